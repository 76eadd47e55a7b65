// The Wilson solver templates (stencils, BiCGStab kernels, the even-odd iteration, the solver
// engine, apply and stencil benchmark), instantiated per iteration precision by
// hp_wilson_fp64.cu, hp_wilson_fp32.cu, hp_wilson_fp16.cu and hp_wilson_bf16.cu so that the four
// precisions compile in parallel; hp_wilson.cu holds the operator preparation and the dispatch.
#pragma once
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hp_fields.cuh"

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

// Stencil variants: slots per sweep group G (0 = all slots in one sweep), right-hand sides per
// thread (1, 2, 4) and link storage (12 or 18 reals), encoded as
// variant = 100 * G + 10 * RPT + (REC == 18).  FP64 always uses full links.
static int variant_rpt(int v) { return (v % 100) / 10; }
static int variant_rec(int v) { return (v % 10) ? 18 : 12; }
static int variant_group(int v) { return v / 100; }
// launch grid of the stencil for nslots slots: (group members, tiles, groups)
static dim3 stencil_grid(int variant, int nslots, int ntiles_y) {
  const int rpt = variant_rpt(variant);
  const int units = (nslots + rpt - 1) / rpt;                 // blocks needed along the slots
  int g = variant_group(variant);
  int gx = g > 0 ? std::max(1, std::min(units, g / rpt)) : units;
  int gz = (units + gx - 1) / gx;
  return dim3(gx, ntiles_y, gz);
}

// Blocks per slot: every tile of the lattice, so one active slot fills the GPU on its own
// (masked launches often carry a single slot).
static int dslash_gridy(hp_ctx* ctx, int V, int NT, int nslots) {
  (void)ctx;
  (void)nslots;
  // one tile per block: blocks are dispatched in index order, so the lattice is swept once in
  // site order and the +-t neighbours of a tile are still in L2 when they are read again
  int ntiles = (V + NT - 1) / NT;
  return std::max(1, std::min(ntiles, 65535));
}

// ==================================================================== solver
// Per slot (right-hand side) BiCGStab, x_0 = 0, shadow r^ = b:
//   v = D p; alpha = rho / (r^, v); s = r - alpha v; t = D s;
//   omega = (t, s) / (t, t); e += alpha p + omega s; r = s - omega t;
//   rho' = (r^, r); beta = (rho'/rho)(alpha/omega); p = r + beta (p - omega v)
// in the iteration precision (FP16/BF16 storage with FP32 arithmetic, or
// FP32), e accumulating the solution since the last update.  Updates:
//   group (FP32):  whenever ||r|| < delta max||r|| since the last update:
//                  r_g -= D e (FP32 links and arithmetic), x += e (FP64),
//                  e = 0, r = r_g.  x and r_g stay consistent whatever the
//                  rounding of e, and the error of D e is ~1e-7 ||r||.
//   exact (FP64):  when ||r|| <= tol ||b|| or ||r|| < 1e-5 of the residual
//                  at the previous exact update: x += e, e = 0,
//                  r = r_g = b - D x with FP64 links and arithmetic; the
//                  solve stops when this true residual is <= tol ||b||.
// FP64 solves run the same iteration in FP64 with exact updates only.
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
  FieldPtr rg;           // group-updated residual (FP32), mixed precision only
  double2* x;            // FP64 solution [slot][12][Vmax] (FP64 solves)
  FieldPtr xff;          // float-float solution (hi, lo FP32 fields), mixed precision
  double tol2, delta2, epsx2;
  int maxiter;
  // even-odd: Krylov fields live on the odd sites (half-site index = site >> 1)
  int eo;
  FieldPtr mid;          // even-site intermediate of the Schur operator (iteration precision)
  FieldPtr mid32;        // even-site intermediate of group updates (FP32)
  double2* xe;           // even-site solution, FP64 solves
  FieldPtr xeff;         // even-site solution, float-float (mixed)
};

#define SLOT_PREAMBLE(COND)                                        \
  const int slot = blockIdx.x;                                     \
  SlotState* S = a.st + slot;                                      \
  if (!(COND)) return;                                             \
  const LatGeom g = a.lats[S->lat];                                \
  const int nsite = a.eo ? (g.V >> 1) : g.V;                       \
  const int ntiles = (nsite + NT - 1) / NT;                        \
  if ((int)blockIdx.y >= ntiles) return;                           \
  const int nparts = min((int)gridDim.y, ntiles);                  \
  double* part = a.part + (size_t)slot * 4 * a.gy;                 \
  (void)nparts;                                                    \
  (void)nsite;                                                     \
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

// diagonal 1 + m + mu(x) in the kernel's arithmetic (FP32 kernels read an FP32 copy of mu)
template <typename R>
__device__ __forceinline__ R site_diag(const LatGeom& g, int site) {
  return (R)g.diag0 + (g.mass_field32 ? (R)g.mass_field32[site] : (R)0);
}
template <>
__device__ __forceinline__ double site_diag<double>(const LatGeom& g, int site) {
  return 1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0);
}

// acc += n * (diagonal term) c: (1 + m + mu(x)) n c, or n A(x) c with the clover term (CL = false:
// the caller knows there is none)
template <typename R, bool CL = true>
__device__ __forceinline__ void add_diag(const LatGeom& g, int site, const cplx<R> (&c)[12], R n,
                                         cplx<R> (&acc)[12]) {
  if (CL && g.clover) {
    cplx<R> ac[12];
    clover_mul<R>(g, false, site, c, ac);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[k].x = fma(n, ac[k].x, acc[k].x);
      acc[k].y = fma(n, ac[k].y, acc[k].y);
    }
    return;
  }
  const R dn = site_diag<R>(g, site) * n;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    acc[k].x = fma(dn, c[k].x, acc[k].x);
    acc[k].y = fma(dn, c[k].y, acc[k].y);
  }
}

// ---- the stencil on RPT right-hand sides per thread
// Thread = one site; it loads (and reconstructs) each of the 8 links of the
// site once and applies it to RPT slots of the same lattice.  Epilogues:
//   EPI_PLAIN  out = D in
//   EPI_V      v = D p ; sigma = (r^, v) ; alpha = rho / sigma
//   EPI_T      t = D s ; omega = (t, s) / (t, t)
enum { EPI_PLAIN = 0, EPI_V = 1, EPI_T = 2 };

// Grid: x = member of a slot group (RPT slots each), y = tile, z = slot group.  Blocks run in
// index order, so a group sweeps the lattice with its slots interleaved per tile (the links of
// a tile are read once per group) and groups follow one another (the +-t neighbours of a tile
// are still in L2 when the sweep of a group reaches them).
template <int SPR, int RPT, int NT, int EPI, int REC, bool CL>
__global__ void __launch_bounds__(NT) k_wds(WArgs a, FieldPtr in, FieldPtr out, int nslots) {
  typedef typename Real_of<SPR>::T R;
  constexpr int LPR = LinkPrecOf<SPR>::v;
  constexpr int NQ = EPI == EPI_V ? 2 : 3;
  const int slot0 = (blockIdx.z * gridDim.x + blockIdx.x) * RPT;
  __shared__ int act_sh[RPT];
  __shared__ int lat_sh;
  if (threadIdx.x == 0) {
    int lat = -1;
    for (int r = 0; r < RPT; ++r) {
      const int sl = slot0 + r;
      int on = 0;
      if (sl < nslots) {
        if (EPI == EPI_PLAIN) {
          on = 1;
          lat = 0;
        } else if (a.st[sl].status == SLOT_RUN) {
          on = 1;
          if (lat < 0) lat = a.st[sl].lat;
        }
      }
      act_sh[r] = on;
    }
    lat_sh = lat;
  }
  __syncthreads();
  const int lat = lat_sh;
  if (lat < 0) return;
  bool act[RPT];
#pragma unroll
  for (int r = 0; r < RPT; ++r) act[r] = act_sh[r] != 0;
  const LatGeom g = a.lats[lat];   // by value: the fields used in the loop stay in registers
  const int ntiles = (g.V + NT - 1) / NT;
  if ((int)blockIdx.y >= ntiles) return;
  const int nparts = min((int)gridDim.y, ntiles);
  R dots[RPT][NQ];
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < NQ; ++q) dots[r][q] = (R)0;
  const R mkap = -(R)g.kappa;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    int x[4], st[4];
    site_coords(g, site, x, st);
    // acc = -kappa * hop, accumulated with FMAs (the half-precision norm folded in)
    cplx<R> acc[RPT][12];
#pragma unroll
    for (int r = 0; r < RPT; ++r)
#pragma unroll
      for (int k = 0; k < 12; ++k) acc[r][k] = {(R)0, (R)0};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int L = g.L[mu];
      const int fw = (x[mu] + 1 == L) ? site - (L - 1) * st[mu] : site + st[mu];
      const int bw = (x[mu] == 0) ? site + (L - 1) * st[mu] : site - st[mu];
      cplx<R> u[9];
      LinkIO<LPR, REC>::load(g, mu, site, u);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (!act[r]) continue;
        cplx<R> psi[12], h[6], w[6];
        R n;
        SpinorIO<SPR>::load_nc_raw(in, a.Vmax, slot0 + r, fw, psi, n);
        if (mu == 0) project<0, -1>(psi, h);
        if (mu == 1) project<1, -1>(psi, h);
        if (mu == 2) project<2, -1>(psi, h);
        if (mu == 3) project<3, -1>(psi, h);
        su3_mul<R, false>(u, h, w);
        const R sc = mkap * n;
        if (mu == 0) accumulate_s<0, -1>(acc[r], w, sc);
        if (mu == 1) accumulate_s<1, -1>(acc[r], w, sc);
        if (mu == 2) accumulate_s<2, -1>(acc[r], w, sc);
        if (mu == 3) accumulate_s<3, -1>(acc[r], w, sc);
      }
      LinkIO<LPR, REC>::load(g, mu, bw, u);
#pragma unroll
      for (int r = 0; r < RPT; ++r) {
        if (!act[r]) continue;
        cplx<R> psi[12], h[6], w[6];
        R n;
        SpinorIO<SPR>::load_nc_raw(in, a.Vmax, slot0 + r, bw, psi, n);
        if (mu == 0) project<0, 1>(psi, h);
        if (mu == 1) project<1, 1>(psi, h);
        if (mu == 2) project<2, 1>(psi, h);
        if (mu == 3) project<3, 1>(psi, h);
        su3_mul<R, true>(u, h, w);
        const R sc = mkap * n;
        if (mu == 0) accumulate_s<0, 1>(acc[r], w, sc);
        if (mu == 1) accumulate_s<1, 1>(acc[r], w, sc);
        if (mu == 2) accumulate_s<2, 1>(acc[r], w, sc);
        if (mu == 3) accumulate_s<3, 1>(acc[r], w, sc);
      }
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (!act[r]) continue;
      cplx<R> c[12];
      R nc;
      SpinorIO<SPR>::load_nc_raw(in, a.Vmax, slot0 + r, site, c, nc);
      add_diag<R, CL>(g, site, c, nc, acc[r]);
      SpinorIO<SPR>::store(out, a.Vmax, slot0 + r, site, acc[r]);
      if (EPI == EPI_V) {
        cplx<R> rh[12];
        SpinorIO<SPR>::load(a.rh, a.Vmax, slot0 + r, site, rh);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          cplx<R> d = cconjmul(rh[k], acc[r][k]);
          dots[r][0] += d.x;
          dots[r][1] += d.y;
        }
      } else if (EPI == EPI_T) {
        R d0 = 0, d1 = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
          cplx<R> d = cconjmul(acc[r][k], c[k]);   // (t, s) with s = nc * c
          d0 += d.x;
          d1 += d.y;
          dots[r][2 % NQ] += acc[r][k].x * acc[r][k].x + acc[r][k].y * acc[r][k].y;
        }
        dots[r][0] += nc * d0;
        dots[r][1] += nc * d1;
      }
    }
  }
  if (EPI == EPI_PLAIN) return;
  // per-slot block partials: warp shuffles in the iteration precision, warps in FP64
  __shared__ double shp[RPT][NQ][NT / 32];
  __shared__ int last_sh[RPT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int r = 0; r < RPT; ++r)
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      R t = dots[r][q];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      if (lane == 0) shp[r][q][warp] = (double)t;
    }
  __syncthreads();
  if (threadIdx.x < RPT * NQ) {
    const int r = threadIdx.x / NQ, q = threadIdx.x % NQ;
    if (act_sh[r]) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += shp[r][q][w];
      a.part[((size_t)(slot0 + r) * 4 + q) * a.gy + blockIdx.y] = t;
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x < RPT) {
    int l = 0;
    if (act_sh[threadIdx.x]) {
      unsigned int t = atomicAdd(a.cnt + slot0 + threadIdx.x, 1u);
      l = (t == (unsigned int)nparts - 1u);
    }
    last_sh[threadIdx.x] = l;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < RPT; ++r) {
    if (!last_sh[r]) continue;
    __threadfence();
    double tot[NQ];
    block_sum_partials<NQ, NT>(a.part + (size_t)(slot0 + r) * 4 * a.gy, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      SlotState* S = a.st + slot0 + r;
      if (EPI == EPI_V) {
        S->alpha = cdiv(S->rho, make_double2(tot[0], tot[1]));
        S->restart = 0;
        if (S->need_update == 3) S->need_update = 0;
      } else {
        S->omega = tot[NQ - 1] > 0.0 ? make_double2(tot[0] / tot[NQ - 1], tot[1] / tot[NQ - 1]) : make_double2(0.0, 0.0);
      }
      S->sloppy_mv += 1;
      a.cnt[slot0 + r] = 0;
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
    if (SPR == PR64) {
      SpinorIO<PR64>::store(FieldPtr{a.x, nullptr, nullptr}, a.Vmax, slot, site, z);
    } else {
      cplx<float> zf[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) zf[k] = {0.f, 0.f};
      SpinorIO<PR32>::store(FieldPtr{a.xff.p, nullptr, nullptr}, a.Vmax, slot, site, zf);
      SpinorIO<PR32>::store(FieldPtr{a.xff.lo, nullptr, nullptr}, a.Vmax, slot, site, zf);
    }
    {
      cplx<typename Real_of<EPR>::T> ze[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) ze[k] = {0, 0};
      SpinorIO<EPR>::store(a.e, a.Vmax, slot, site, ze);
    }
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, b);
    SpinorIO<SPR>::store(a.rh, a.Vmax, slot, site, b);
    SpinorIO<SPR>::store(a.p, a.Vmax, slot, site, b);
    if (SPR != PR64) {
      cplx<float> bf[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) bf[k] = {(float)b[k].x, (float)b[k].y};
      SpinorIO<PR32>::store(a.rg, a.Vmax, slot, site, bf);
    }
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
      S->rexact2 = tot[0];
      S->gupdates = 0;
      S->status = tot[0] > 0.0 ? SLOT_RUN : SLOT_DONE;
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
    if (site >= nsite) continue;
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
    if (site >= nsite) continue;
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
        S->need_update = 2;
      } else if (rr <= a.tol2 * S->bnorm2 || rr < a.epsx2 * S->rexact2 || !(rr == rr)) {
        S->need_update = 2;
      } else if (rr < a.delta2 * S->rmax2) {
        S->need_update = 1;
      }
      a.cnt[slot] = 0;
    }
  }
}

// ---- group update (FP32): r_g -= D e ; r = r_g ; (r^, r), ||r||^2   (x += e follows)
template <int SPR, int EPR, int NT>
__global__ void __launch_bounds__(NT) k_grp_update(WArgs a) {
  SLOT_PREAMBLE(S->need_update == 1)
  typedef typename Real_of<SPR>::T R;
  float acc[3] = {0.f, 0.f, 0.f};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    cplx<float> de[12], c[12], rg[12];
    wilson_site<EPR, PR32, float>(g, a.e, a.Vmax, slot, site, de, c);
    SpinorIO<PR32>::load(a.rg, a.Vmax, slot, site, rg);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      rg[k].x -= de[k].x;
      rg[k].y -= de[k].y;
    }
    SpinorIO<PR32>::store(a.rg, a.Vmax, slot, site, rg);
    cplx<R> rs[12], rh[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) rs[k] = {(R)rg[k].x, (R)rg[k].y};
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, rs);
    SpinorIO<SPR>::load(a.rh, a.Vmax, slot, site, rh);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[0] += rg[k].x * rg[k].x + rg[k].y * rg[k].y;
      acc[1] += (float)rh[k].x * rg[k].x + (float)rh[k].y * rg[k].y;
      acc[2] += (float)rh[k].x * rg[k].y - (float)rh[k].y * rg[k].x;
    }
  }
  reduce_partials<float, 3, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      const double rr = tot[0];
      S->rnorm2 = rr;
      S->rmax2 = rr;
      S->rho = S->restart ? make_double2(rr, 0.0) : make_double2(tot[1], tot[2]);
      S->gupdates += 1;
      // 3: group update done, x += e pending (k_ru_accum); cleared by the next k_bicg_v
      S->need_update = (rr <= a.tol2 * S->bnorm2 || rr < a.epsx2 * S->rexact2) ? 2 : 3;
      a.cnt[slot] = 0;
    }
  }
}

// ---- reliable update, part 1: x += e ; e = 0
// FP64 solves keep x in FP64; mixed solves keep x in float-float (hi, lo FP32 fields)
template <int SPR, int EPR, int NT>
__global__ void __launch_bounds__(NT) k_ru_accum(WArgs a) {
  SLOT_PREAMBLE(S->need_update)
  typedef typename Real_of<EPR>::T RE;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= nsite) continue;
    cplx<RE> e[12];
    SpinorIO<EPR>::load(a.e, a.Vmax, slot, site, e);
    if (SPR == PR64) {
      FieldPtr xf{a.x, nullptr, nullptr};
      cplx<double> x[12];
      SpinorIO<PR64>::load(xf, a.Vmax, slot, site, x);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        x[k].x += (double)e[k].x;
        x[k].y += (double)e[k].y;
      }
      SpinorIO<PR64>::store(xf, a.Vmax, slot, site, x);
    } else {
      cplx<ffl> x[12];
      SpinorIO<PRFF>::load(a.xff, a.Vmax, slot, site, x);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        x[k].x += ffl((float)e[k].x);
        x[k].y += ffl((float)e[k].y);
      }
      SpinorIO<PRFF>::store(a.xff, a.Vmax, slot, site, x);
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = {(RE)0, (RE)0};
    SpinorIO<EPR>::store(a.e, a.Vmax, slot, site, e);
  }
}

// finalize of a true residual (both arithmetics)
__device__ __forceinline__ void ru_finalize(WArgs& a, SlotState* S, const double (&tot)[3], int slot) {
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
      S->rexact2 = rr;
      S->rho = S->restart ? make_double2(rr, 0.0) : make_double2(tot[1], tot[2]);
    }
  }
  a.cnt[slot] = 0;
}

// ---- reliable update, part 2: the true residual r = b - D x, stored in the iteration precision
// (and in the FP32 group residual).  FP64 solves: FP64 links and arithmetic.  Mixed solves:
// float-float links, solution and arithmetic on the FP32 pipes (48-bit significand: the
// rounding error of b - D x is ~1e-14 ||b||, far below any tolerance the solver certifies).
template <int SPR, int NT>
__global__ void __launch_bounds__(NT, 3) k_ru_residual(WArgs a) {
  SLOT_PREAMBLE(S->need_update == 2)
  typedef typename Real_of<SPR>::T R;
  const int comp = S->a, m = S->m;
  if (SPR == PR64) {
    double acc[3] = {0.0, 0.0, 0.0};
    FieldPtr xf{a.x, nullptr, nullptr};
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
  } else {
    float acc[3] = {0.f, 0.f, 0.f};
    for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
      const int site = tile * NT + threadIdx.x;
      if (site >= g.V) continue;
      cplx<ffl> o[12], c[12];
      wilson_site<PRFF, PRFF, ffl>(g, a.xff, a.Vmax, slot, site, o, c);
      double2 bv = source_value(g, site, m);
      cplx<float> rf[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        ffl rx = -o[k].x, ry = -o[k].y;
        if (k == comp) {
          rx += ffl(bv.x);
          ry += ffl(bv.y);
        }
        rf[k] = {rx.hi, ry.hi};
      }
      cplx<R> rs[12], rh[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) rs[k] = {(R)rf[k].x, (R)rf[k].y};
      SpinorIO<SPR>::store(a.r, a.Vmax, slot, site, rs);
      SpinorIO<PR32>::store(a.rg, a.Vmax, slot, site, rf);
      SpinorIO<SPR>::load(a.rh, a.Vmax, slot, site, rh);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        acc[0] += rf[k].x * rf[k].x + rf[k].y * rf[k].y;
        acc[1] += (float)rh[k].x * rf[k].x + (float)rh[k].y * rf[k].y;
        acc[2] += (float)rh[k].x * rf[k].y - (float)rh[k].y * rf[k].x;
      }
    }
    reduce_partials<float, 3, NT>(acc, part, a.gy);
  }
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) ru_finalize(a, S, tot, slot);
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
    if (site >= nsite) continue;
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
// one component of the converged solution in FP64 (from FP64 or float-float storage)
__device__ __forceinline__ double2 solution_component(const WArgs& a, int slot, int site, int comp) {
  if (a.x) return a.x[((size_t)slot * 12 + comp) * a.Vmax + site];
  const size_t off = ((size_t)slot * 6 + comp / 2) * a.Vmax + site;
  const float4 h = ((const float4*)a.xff.p)[off], l = ((const float4*)a.xff.lo)[off];
  return (comp & 1) ? make_double2((double)h.z + (double)l.z, (double)h.w + (double)l.w)
                    : make_double2((double)h.x + (double)l.x, (double)h.y + (double)l.y);
}

template <int NT>
__global__ void __launch_bounds__(NT) k_quad(WArgs a) {
  SLOT_PREAMBLE(S->status == SLOT_DONE || S->status == SLOT_FAIL)
  double acc[2] = {0.0, 0.0};
  const int comp = S->a, m = S->m;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double2 bv = source_value(g, site, m);
    const double2 xv = solution_component(a, slot, site, comp);
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
static __global__ void k_w_grad(WArgs a, int lat, const int* __restrict__ slots, int nsl, double* __restrict__ grad, int V) {
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < V; site += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nsl; ++i) {
      const int slot = slots[i];
      const SlotState* S = a.st + slot;
      if (S->lat != lat) continue;
      const double sa = S->a < 6 ? 1.0 : -1.0;
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double2 v = solution_component(a, slot, site, k);
        t += (k < 6 ? 1.0 : -1.0) * (v.x * v.x + v.y * v.y);
      }
      acc += sa * t;
    }
    grad[site] += acc;
  }
}

// ============================================================= even-odd (Schur)
// With d(x) = 1 + m + mu(x) and H the hopping term, D = [[d_e, -k H_eo], [-k H_oe, d_o]].
// The odd-site Schur complement  S = d_o - k^2 H_oe d_e^-1 H_eo  is solved for x_o; the even
// half follows as x_e = d_e^-1 (b_e + k H_eo x_o), and then the odd part of the full residual
// is  r_o = b_o - d_o x_o + k H_oe x_e  while the even part vanishes by construction: the
// certified residual is the residual of the full system.  Sites of one parity are numbered
// by site >> 1 (every extent even: otherwise some hop joins sites of one parity and the split fails).
enum { MASK_RUN = 0, MASK_GROUP = 1, MASK_EXACT = 2, MASK_FRESH = 3 };

__device__ __forceinline__ bool eo_mask(const SlotState* S, int mask) {
  if (mask == MASK_RUN) return S->status == SLOT_RUN;
  if (mask == MASK_GROUP) return S->need_update == 1;
  if (mask == MASK_FRESH) return S->status == SLOT_RUN && S->restart == 2 && S->need_update == 0;
  return S->need_update == 2;
}

// full index and coordinates of half-site h of parity `par`
__device__ __forceinline__ int eo_site(const LatGeom& g, int h, int par, int (&x)[4], int (&st)[4]) {
  const int l1h = g.L[0] >> 1;
  const int x1h = h % l1h;
  int rest = h / l1h;
  x[1] = rest % g.L[1];
  rest /= g.L[1];
  x[2] = rest % g.L[2];
  x[3] = rest / g.L[2];
  x[0] = 2 * x1h + ((par + x[1] + x[2] + x[3]) & 1);
  st[0] = 1;
  st[1] = g.L[0];
  st[2] = g.L[0] * g.L[1];
  st[3] = st[2] * g.L[2];
  return x[0] + st[1] * x[1] + st[2] * x[2] + st[3] * x[3];
}

// acc += sc * hop(in) at full site `site`, `in` a half-lattice field of the other parity
template <int SPR, int LPR, int REC, typename R>
__device__ __forceinline__ void eo_hop(const LatGeom& g, FieldPtr in, int Vs, int slot, int site, const int (&x)[4],
                                       const int (&st)[4], R sc, cplx<R> (&acc)[12]) {
  if constexpr (is_ffl<R>::value) {   // float-float fields (norm 1): acc += sc hop
    cplx<ffl> t[12];
    hop_ff<SPR, LPR, REC, true>(g, in, Vs, slot, site, x, st, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[k].x = fma(sc, t[k].x, acc[k].x);
      acc[k].y = fma(sc, t[k].y, acc[k].y);
    }
    return;
  }
#pragma unroll
  for (int mu = 0; mu < 4; ++mu) {
    const int L = g.L[mu];
    const int fw = (x[mu] + 1 == L) ? site - (L - 1) * st[mu] : site + st[mu];
    const int bw = (x[mu] == 0) ? site + (L - 1) * st[mu] : site - st[mu];
    cplx<R> u[9], psi[12], h[6], w[6];
    R n;
    LinkIO<LPR, REC>::load(g, mu, site, u);
    SpinorIO<SPR>::load_nc_raw(in, Vs, slot, fw >> 1, psi, n);
    if (mu == 0) project<0, -1>(psi, h);
    if (mu == 1) project<1, -1>(psi, h);
    if (mu == 2) project<2, -1>(psi, h);
    if (mu == 3) project<3, -1>(psi, h);
    su3_mul<R, false>(u, h, w);
    if (mu == 0) accumulate_s<0, -1>(acc, w, sc * n);
    if (mu == 1) accumulate_s<1, -1>(acc, w, sc * n);
    if (mu == 2) accumulate_s<2, -1>(acc, w, sc * n);
    if (mu == 3) accumulate_s<3, -1>(acc, w, sc * n);
    LinkIO<LPR, REC>::load(g, mu, bw, u);
    SpinorIO<SPR>::load_nc_raw(in, Vs, slot, bw >> 1, psi, n);
    if (mu == 0) project<0, 1>(psi, h);
    if (mu == 1) project<1, 1>(psi, h);
    if (mu == 2) project<2, 1>(psi, h);
    if (mu == 3) project<3, 1>(psi, h);
    su3_mul<R, true>(u, h, w);
    if (mu == 0) accumulate_s<0, 1>(acc, w, sc * n);
    if (mu == 1) accumulate_s<1, 1>(acc, w, sc * n);
    if (mu == 2) accumulate_s<2, 1>(acc, w, sc * n);
    if (mu == 3) accumulate_s<3, 1>(acc, w, sc * n);
  }
}

__device__ __forceinline__ double leading_part(double v) { return v; }
__device__ __forceinline__ double leading_part(ffl v) { return (double)v.hi; }

// The slots of an even-odd launch.  LOOP = false: one slot per block (grid x/z: the slot, y: the
// tile), for launches that serve most slots; LOOP = true: one block per tile (grid 1 x tiles) that
// loops over the slots its mask selects, for launches that serve a few slots at a time (the exact
// and group steps, fresh starts): an unselected slot then costs a flag test, not a block.  Every
// block of a tile reads a slot's mask before that slot's finalisation (the last block to finish
// it), so the loop is uniform over the block.
#define EO_SLOTS_BEGIN(MASK, LOOP)                                                  \
  const int s_first = (LOOP) ? 0 : (int)(blockIdx.z * gridDim.x + blockIdx.x);     \
  const int s_last = (LOOP) ? nslots : min(s_first + 1, nslots);                    \
  for (int slot = s_first; slot < s_last; ++slot) {                                 \
    SlotState* S = a.st + slot;                                                     \
    if (!eo_mask(S, MASK)) continue;                                                \
    const LatGeom g = a.lats[S->lat];                                               \
    const int nsite = g.V >> 1;                                                     \
    const int ntiles = (nsite + NT - 1) / NT;                                       \
    if ((int)blockIdx.y >= ntiles) continue;                                        \
    const int nparts = min((int)gridDim.y, ntiles);                                 \
    double* part = a.part + (size_t)slot * 4 * a.gy;                                \
    (void)nparts;                                                                   \
    (void)part;
#define EO_SLOTS_END }

// ---- even sites: mid = d_e^-1 hop(in_o)  (register caps: six resident blocks, <= 85 registers, for
// the iteration's launches -- left alone the compiler takes 160 and halves the warps; four for the
// group update)
template <int SIN, int LPR, int REC, int SOUT, int NT, int MASK, bool CL>
__global__ void __launch_bounds__(NT, SIN == PR64 ? 2 : (MASK == MASK_RUN ? 6 : 4)) k_eo_even(WArgs a, FieldPtr in, FieldPtr mid, int nslots) {
  EO_SLOTS_BEGIN(MASK, MASK != MASK_RUN)
  typedef typename Real_of<SIN>::T R;   // FP64 for the FP64 solver, FP32 arithmetic otherwise
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 0, x, st);
    if constexpr (CL) {
      if (g.clover) {   // A_e(x)^-1 hop
        cplx<R> acc[12], t[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = {(R)0, (R)0};
        eo_hop<SIN, LPR, REC, R>(g, in, a.Vmax, slot, site, x, st, (R)1, acc);
        clover_mul<R>(g, true, site, acc, t);
        SpinorIO<SOUT>::store(mid, a.Vmax, slot, h, t);
        continue;
      }
    }
    const R inv = (R)1 / site_diag<R>(g, site);
    cplx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {(R)0, (R)0};
    eo_hop<SIN, LPR, REC, R>(g, in, a.Vmax, slot, site, x, st, inv, acc);
    SpinorIO<SOUT>::store(mid, a.Vmax, slot, h, acc);
  }
  EO_SLOTS_END
}

// ---- odd sites: out = d_o in - k^2 hop(mid), with the solver epilogues
//   EPI_V: v = S p, (r^, v), alpha       EPI_T: t = S s, (t, s), (t, t), omega
//   EPI_G: group update r_g -= S e, r = r_g, (r^, r_g), ||r_g||^2   (in = e, mid FP32)
enum { EPI_G = 3 };

// resident blocks of 128 threads: six (<= 85 registers) with 18-real links, five (<= 102) with the
// reconstructing 12-real form; the odd-site kernels are latency-bound, and the register count the
// compiler picks unconstrained halves the warps an SM holds; the FP64 solver's FP64 arithmetic gets two
// (<= 256 registers: its twelve complex accumulators alone take 48)
#define EO_ODD_MINB(SIN, REC) ((SIN) == PR64 ? 2 : (REC) == 18 ? 6 : 5)
template <int SIN, int SMID, int LPR, int REC, int NT, int EPI, bool CL>
__global__ void __launch_bounds__(NT, EO_ODD_MINB(SIN, REC)) k_eo_odd(WArgs a, FieldPtr in, FieldPtr mid, FieldPtr out, int nslots) {
  EO_SLOTS_BEGIN(EPI == EPI_G ? MASK_GROUP : MASK_RUN, EPI == EPI_G)
  typedef typename Real_of<SIN>::T R;   // FP64 for the FP64 solver, FP32 arithmetic otherwise
  constexpr int NQ = EPI == EPI_V ? 2 : 3;
  R dots[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) dots[q] = (R)0;
  const R mk2 = -(R)(g.kappa * g.kappa);
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 1, x, st);
    cplx<R> acc[12], c[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {(R)0, (R)0};
    eo_hop<SMID, LPR, REC, R>(g, mid, a.Vmax, slot, site, x, st, mk2, acc);
    R nc;
    SpinorIO<SIN>::load_nc_raw(in, a.Vmax, slot, h, c, nc);
    add_diag<R, CL>(g, site, c, nc, acc);
    if (EPI == EPI_G) {
      cplx<R> rg[12], rh[12];
      SpinorIO<PR32>::load(a.rg, a.Vmax, slot, h, rg);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        rg[k].x -= acc[k].x;
        rg[k].y -= acc[k].y;
      }
      SpinorIO<PR32>::store(a.rg, a.Vmax, slot, h, rg);
      SpinorIO<SIN>::store(a.r, a.Vmax, slot, h, rg);
      SpinorIO<SIN>::load(a.rh, a.Vmax, slot, h, rh);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        dots[0] += rg[k].x * rg[k].x + rg[k].y * rg[k].y;
        dots[1] += rh[k].x * rg[k].x + rh[k].y * rg[k].y;
        dots[2 % NQ] += rh[k].x * rg[k].y - rh[k].y * rg[k].x;
      }
      continue;
    }
    SpinorIO<SIN>::store(out, a.Vmax, slot, h, acc);
    if (EPI == EPI_V) {
      cplx<R> rh[12];
      SpinorIO<SIN>::load(a.rh, a.Vmax, slot, h, rh);
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cplx<R> d = cconjmul(rh[k], acc[k]);
        dots[0] += d.x;
        dots[1] += d.y;
      }
    } else {
      R d0 = 0, d1 = 0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        cplx<R> d = cconjmul(acc[k], c[k]);
        d0 += d.x;
        d1 += d.y;
        dots[2 % NQ] += acc[k].x * acc[k].x + acc[k].y * acc[k].y;
      }
      dots[0] += nc * d0;
      dots[1] += nc * d1;
    }
  }
  reduce_partials<R, NQ, NT>(dots, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[NQ];
    block_sum_partials<NQ, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      if (EPI == EPI_V) {
        S->alpha = cdiv(S->rho, make_double2(tot[0], tot[1]));
        S->restart = 0;
        if (S->need_update == 3) S->need_update = 0;
        S->sloppy_mv += 1;
      } else if (EPI == EPI_T) {
        S->omega = tot[NQ - 1] > 0.0 ? make_double2(tot[0] / tot[NQ - 1], tot[1] / tot[NQ - 1]) : make_double2(0.0, 0.0);
        S->sloppy_mv += 1;
      } else {
        const double rr = tot[0];
        S->rnorm2 = rr;
        S->rmax2 = rr;
        S->rho = S->restart ? make_double2(rr, 0.0) : make_double2(tot[1], tot[2]);
        S->gupdates += 1;
        S->need_update = (rr <= a.tol2 * S->bnorm2 || rr < a.epsx2 * S->rexact2) ? 2 : 3;
      }
      a.cnt[slot] = 0;
    }
  }
  EO_SLOTS_END
}

// the exact steps: resident blocks of 128 threads (register caps, chosen by timing on 32^3x64):
// step 1 at 3 (168 registers), the float-float step 2 at 2 (its hop plus the residual epilogue
// spills at 168; without spills it runs 13% faster)
#define EO_X_MINB 3
#define EO_X2_MINB 2
// ---- exact step 1: x_e = d_e^-1 (b_e + k hop(x_o))   (FP64 or float-float)
template <int PX, int NT>
__global__ void __launch_bounds__(NT, EO_X_MINB) k_eo_x1(WArgs a, int nslots) {
  EO_SLOTS_BEGIN(MASK_EXACT, true)
  typedef typename Real_of<PX>::T R;
  const int comp = S->a, m = S->m;
  FieldPtr xo = PX == PR64 ? FieldPtr{a.x, nullptr, nullptr} : a.xff;
  FieldPtr xe = PX == PR64 ? FieldPtr{a.xe, nullptr, nullptr} : a.xeff;
  const R kap = R(g.kappa);
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 0, x, st);
    cplx<R> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    eo_hop<PX, PX, 12, R>(g, xo, a.Vmax, slot, site, x, st, kap, acc);
    const double2 bv = source_value(g, site, m);
#pragma unroll
    for (int k = 0; k < 12; ++k)
      if (k == comp) {
        acc[k].x = acc[k].x + R(bv.x);
        acc[k].y = acc[k].y + R(bv.y);
      }
    if (g.clover) {   // A_e(x)^-1 (b_e + k hop)
      cplx<R> t[12];
      clover_mul<R>(g, true, site, acc, t);
      SpinorIO<PX>::store(xe, a.Vmax, slot, h, t);
      continue;
    }
    const R inv = R(1.0 / (1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0)));
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      acc[k].x = inv * acc[k].x;
      acc[k].y = inv * acc[k].y;
    }
    SpinorIO<PX>::store(xe, a.Vmax, slot, h, acc);
  }
  EO_SLOTS_END
}

// ---- exact step 2: r_o = b_o - d_o x_o + k hop(x_e); a fresh slot also sets r^ = p = r
template <int SPR, int PX, int NT>
__global__ void __launch_bounds__(NT, PX == PR64 ? EO_X_MINB : EO_X2_MINB) k_eo_x2(WArgs a, int nslots) {
  EO_SLOTS_BEGIN(MASK_EXACT, true)
  typedef typename Real_of<PX>::T R;
  typedef typename Real_of<SPR>::T RS;
  const int comp = S->a, m = S->m;
  const bool fresh = S->restart == 2;
  FieldPtr xo = PX == PR64 ? FieldPtr{a.x, nullptr, nullptr} : a.xff;
  FieldPtr xe = PX == PR64 ? FieldPtr{a.xe, nullptr, nullptr} : a.xeff;
  const R kap = R(g.kappa);
  float acc3[3] = {0.f, 0.f, 0.f};
  double accd[3] = {0.0, 0.0, 0.0};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 1, x, st);
    cplx<R> acc[12], c[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {R(0), R(0)};
    eo_hop<PX, PX, 12, R>(g, xe, a.Vmax, slot, site, x, st, kap, acc);
    SpinorIO<PX>::load_nc(xo, a.Vmax, slot, h, c);
    if (g.clover) {   // c := A_o(x) x_o, subtracted below with d = 1
      cplx<R> t[12];
      clover_mul<R>(g, false, site, c, t);
#pragma unroll
      for (int k = 0; k < 12; ++k) c[k] = t[k];
    }
    const R d = g.clover ? R(1.0) : R(1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0));
    const double2 bv = source_value(g, site, m);
    cplx<RS> rs[12];
    cplx<float> rf[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      R rx = acc[k].x - d * c[k].x, ry = acc[k].y - d * c[k].y;
      if (k == comp) {
        rx = rx + R(bv.x);
        ry = ry + R(bv.y);
      }
      const double dx = leading_part(rx), dy = leading_part(ry);
      rs[k] = {(RS)dx, (RS)dy};
      rf[k] = {(float)dx, (float)dy};
    }
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, h, rs);
    if (PX != PR64) SpinorIO<PR32>::store(a.rg, a.Vmax, slot, h, rf);
    if (fresh) {
      SpinorIO<SPR>::store(a.rh, a.Vmax, slot, h, rs);
      SpinorIO<SPR>::store(a.p, a.Vmax, slot, h, rs);
    }
    cplx<RS> rh[12];
    SpinorIO<SPR>::load(a.rh, a.Vmax, slot, h, rh);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (PX == PR64) {
        accd[0] += (double)rs[k].x * rs[k].x + (double)rs[k].y * rs[k].y;
        accd[1] += (double)rh[k].x * rs[k].x + (double)rh[k].y * rs[k].y;
        accd[2] += (double)rh[k].x * rs[k].y - (double)rh[k].y * rs[k].x;
      } else {
        acc3[0] += rf[k].x * rf[k].x + rf[k].y * rf[k].y;
        acc3[1] += (float)rh[k].x * rf[k].x + (float)rh[k].y * rf[k].y;
        acc3[2] += (float)rh[k].x * rf[k].y - (float)rh[k].y * rf[k].x;
      }
    }
  }
  if (PX == PR64) reduce_partials<double, 3, NT>(accd, part, a.gy);
  else reduce_partials<float, 3, NT>(acc3, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[3];
    block_sum_partials<3, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      if (fresh) {   // initial residual of the Schur system: start the iteration from it
        S->restart = 0;
        S->need_update = 0;
        S->rnorm2 = S->rmax2 = S->rexact2 = tot[0];
        S->rho = make_double2(tot[0], 0.0);
        S->true_res2 = tot[0];
        if (!(tot[0] > a.tol2 * S->bnorm2)) S->status = SLOT_DONE;
        a.cnt[slot] = 0;
      } else {
        ru_finalize(a, S, tot, slot);
      }
    }
  }
  EO_SLOTS_END
}

// ---- init: x_o = 0, e = 0, ||b||^2 over the whole lattice; the exact steps then set
// x_e = d_e^-1 b_e and r = r^ = p = b_o + k H_oe x_e
template <int SPR, int EPR, int NT>
__global__ void __launch_bounds__(NT) k_eo_init(WArgs a, int nslots) {
  const int slot = blockIdx.x;
  if (slot >= nslots) return;
  SlotState* S = a.st + slot;
  if (S->status != SLOT_INIT) return;
  const LatGeom g = a.lats[S->lat];
  const int ntiles = (g.V + NT - 1) / NT;
  if ((int)blockIdx.y >= ntiles) return;
  const int nparts = min((int)gridDim.y, ntiles);
  double* part = a.part + (size_t)slot * 4 * a.gy;
  const int m = S->m;
  double acc[1] = {0.0};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    const double2 bv = source_value(g, site, m);
    acc[0] += bv.x * bv.x + bv.y * bv.y;
    const int h = site >> 1;
    int r = site, par = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      par += r % g.L[j];
      r /= g.L[j];
    }
    if ((par & 1) == 0) {           // odd sites carry the Krylov vectors
      if (SPR != PR64) {            // x_e = 0 until the first exact step (the mixed start skips it)
        cplx<float> z[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = {0.f, 0.f};
        SpinorIO<PR32>::store(FieldPtr{a.xeff.p, nullptr, nullptr}, a.Vmax, slot, h, z);
        SpinorIO<PR32>::store(FieldPtr{a.xeff.lo, nullptr, nullptr}, a.Vmax, slot, h, z);
      }
      continue;
    }
    cplx<typename Real_of<EPR>::T> ze[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ze[k] = {0, 0};
    SpinorIO<EPR>::store(a.e, a.Vmax, slot, h, ze);
    if (SPR == PR64) {
      cplx<double> z[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) z[k] = {0.0, 0.0};
      SpinorIO<PR64>::store(FieldPtr{a.x, nullptr, nullptr}, a.Vmax, slot, h, z);
    } else {
      cplx<float> z[12];
#pragma unroll
      for (int k = 0; k < 12; ++k) z[k] = {0.f, 0.f};
      SpinorIO<PR32>::store(FieldPtr{a.xff.p, nullptr, nullptr}, a.Vmax, slot, h, z);
      SpinorIO<PR32>::store(FieldPtr{a.xff.lo, nullptr, nullptr}, a.Vmax, slot, h, z);
    }
  }
  reduce_partials<double, 1, NT>(acc, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->bnorm2 = tot[0];
      S->alpha = make_double2(1.0, 0.0);
      S->omega = make_double2(1.0, 0.0);
      S->beta = make_double2(0.0, 0.0);
      S->iters = 0;
      S->updates = 0;
      S->sloppy_mv = 0;
      S->fp64_mv = 0;
      S->gupdates = 0;
      S->restart = 2;          // fresh: the start kernels produce the initial residual
      S->need_update = SPR == PR64 ? 2 : 0;   // FP64: the exact steps; mixed: the FP32 start
      S->status = tot[0] > 0.0 ? SLOT_RUN : SLOT_DONE;
      a.cnt[slot] = 0;
    }
  }
}

// ---- mixed-precision start (FP32), in place of the exact steps of the FP64 mode:
//   mid32 = d_e^-1 b_e on the even sites, then r = r^ = p = r_g = b_o + k H_oe mid32.
// The initial residual only seeds the iteration (every exact step recomputes the residual from
// x, and x_e from x_o), so FP32 accuracy suffices here.  A start residual at or below the
// tolerance is handed to the exact steps, which certify or continue it.
template <int NT>
__global__ void __launch_bounds__(NT) k_eo_src(WArgs a, int nslots) {
  EO_SLOTS_BEGIN(MASK_FRESH, true)
  const int comp = S->a, m = S->m;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 0, x, st);
    const double2 bv = source_value(g, site, m);
    const float inv = g.clover ? 1.0f : 1.0f / site_diag<float>(g, site);
    cplx<float> z[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) z[k] = k == comp ? cplx<float>{inv * (float)bv.x, inv * (float)bv.y}
                                                   : cplx<float>{0.f, 0.f};
    if (g.clover) {   // A_e(x)^-1 b_e
      cplx<float> t[12];
      clover_mul<float>(g, true, site, z, t);
      SpinorIO<PR32>::store(a.mid32, a.Vmax, slot, h, t);
      continue;
    }
    SpinorIO<PR32>::store(a.mid32, a.Vmax, slot, h, z);
  }
  EO_SLOTS_END
}

template <int SPR, int NT>
__global__ void __launch_bounds__(NT) k_eo_r0(WArgs a, int nslots) {
  EO_SLOTS_BEGIN(MASK_FRESH, true)
  typedef typename Real_of<SPR>::T RS;
  const int comp = S->a, m = S->m;
  const float kap = (float)g.kappa;
  float acc1[1] = {0.f};
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int h = tile * NT + threadIdx.x;
    if (h >= nsite) continue;
    int x[4], st[4];
    const int site = eo_site(g, h, 1, x, st);
    cplx<float> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.f, 0.f};
    eo_hop<PR32, PR32, 12, float>(g, a.mid32, a.Vmax, slot, site, x, st, kap, acc);
    const double2 bv = source_value(g, site, m);
    cplx<RS> rs[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      if (k == comp) {
        acc[k].x += (float)bv.x;
        acc[k].y += (float)bv.y;
      }
      rs[k] = {(RS)acc[k].x, (RS)acc[k].y};
      acc1[0] += acc[k].x * acc[k].x + acc[k].y * acc[k].y;
    }
    SpinorIO<PR32>::store(a.rg, a.Vmax, slot, h, acc);
    SpinorIO<SPR>::store(a.r, a.Vmax, slot, h, rs);
    SpinorIO<SPR>::store(a.rh, a.Vmax, slot, h, rs);
    SpinorIO<SPR>::store(a.p, a.Vmax, slot, h, rs);
  }
  reduce_partials<float, 1, NT>(acc1, part, a.gy);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      if (tot[0] > a.tol2 * S->bnorm2) {
        S->restart = 0;
        S->rnorm2 = S->rmax2 = S->rexact2 = tot[0];
        S->rho = make_double2(tot[0], 0.0);
        S->true_res2 = tot[0];
      } else {
        S->need_update = 2;   // still fresh: the exact steps start (or finish) this slot
      }
      a.cnt[slot] = 0;
    }
  }
  EO_SLOTS_END
}

// one component of the converged solution at a full site, from the parity fields
__device__ __forceinline__ double2 eo_solution_component(const WArgs& a, int slot, int site, int par, int comp) {
  const int h = site >> 1;
  if (a.x) {
    const double2* f = par ? a.x : a.xe;
    return f[((size_t)slot * 12 + comp) * a.Vmax + h];
  }
  const FieldPtr f = par ? a.xff : a.xeff;
  const size_t off = ((size_t)slot * 6 + comp / 2) * a.Vmax + h;
  const float4 hi = ((const float4*)f.p)[off], lo = ((const float4*)f.lo)[off];
  return (comp & 1) ? make_double2((double)hi.z + (double)lo.z, (double)hi.w + (double)lo.w)
                    : make_double2((double)hi.x + (double)lo.x, (double)hi.y + (double)lo.y);
}

__device__ __forceinline__ int site_parity(const LatGeom& g, int site) {
  int r = site, par = 0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    par += r % g.L[j];
    r /= g.L[j];
  }
  return par & 1;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_eo_quad(WArgs a, int nslots) {
  const int slot = blockIdx.x;
  if (slot >= nslots) return;
  SlotState* S = a.st + slot;
  if (!(S->status == SLOT_DONE || S->status == SLOT_FAIL)) return;
  const LatGeom g = a.lats[S->lat];
  const int ntiles = (g.V + NT - 1) / NT;
  if ((int)blockIdx.y >= ntiles) return;
  const int nparts = min((int)gridDim.y, ntiles);
  double* part = a.part + (size_t)slot * 4 * a.gy;
  double acc[2] = {0.0, 0.0};
  const int comp = S->a, m = S->m;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    const double2 bv = source_value(g, site, m);
    const double2 xv = eo_solution_component(a, slot, site, site_parity(g, site), comp);
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

static __global__ void k_eo_grad(WArgs a, int lat, const int* __restrict__ slots, int nsl, double* __restrict__ grad,
                          LatGeom g) {
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < g.V; site += gridDim.x * blockDim.x) {
    const int par = site_parity(g, site);
    double acc = 0.0;
    for (int i = 0; i < nsl; ++i) {
      const int slot = slots[i];
      const SlotState* S = a.st + slot;
      if (S->lat != lat) continue;
      const double sa = S->a < 6 ? 1.0 : -1.0;
      double t = 0.0;
#pragma unroll
      for (int k = 0; k < 12; ++k) {
        const double2 v = eo_solution_component(a, slot, site, par, k);
        t += (k < 6 ? 1.0 : -1.0) * (v.x * v.x + v.y * v.y);
      }
      acc += sa * t;
    }
    grad[site] += acc;
  }
}

// ---- the solutions of harvested slots in the canonical layout: slot slots[i] -> right-hand side idx[i]
// of out (complex [n][V][12]; FP64, float-float hi + lo, or the two parities of the even-odd iteration)
static __global__ void k_w_keep(WArgs a, const int* __restrict__ slots, const int* __restrict__ idx, int nsl,
                                double2* __restrict__ out, LatGeom g) {
  const long long total = (long long)nsl * g.V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(t / g.V), site = (int)(t - (long long)i * g.V);
    const int slot = slots[i];
    double2* o = out + ((size_t)idx[i] * g.V + site) * 12;
    const int par = a.eo ? site_parity(g, site) : 0;
#pragma unroll
    for (int k = 0; k < 12; ++k)
      o[k] = a.eo ? eo_solution_component(a, slot, site, par, k) : solution_component(a, slot, site, k);
  }
}

// the even-odd V and T steps with two right-hand sides per thread (FP16 / BF16 / FP32 iteration)
#include "hp_eo2.cuh"
#include "hp_eo3.cuh"

// ================================================================ the engine
template <int SPR>
static hp_status tune_rpt(hp_ctx* ctx, const LatGeom& g, FieldPtr fi, FieldPtr fo, int nrhs, int Vmax, int* best);
template <int SPR>
__global__ void k_w_fill(FieldPtr f, int V, int nrhs, unsigned long long seed);

template <int SPR>
struct WilsonEngine {
  static constexpr int EPR = SPR;      // solution increment e kept in the iteration precision
  static constexpr int NT = 128;
  static constexpr int GROUP_MAX = 4;
  static constexpr int PX = SPR == PR64 ? PR64 : PRFF;   // arithmetic of the true residual
  hp_ctx* ctx;
  bool eo = false;     // even-odd (Schur complement) iteration; set before setup
  bool clover = false; // some lattice of the problem carries the clover term; set before setup
  WArgs a;
  int nslots, gy, gyb, rpt = 1, variant = 10;
  int eo_kernel = 4;   // even-odd V / T steps: 1 one right-hand side per thread, 10 L + B pair kernels
                       // (B = 3 or 4 resident blocks per SM, L = 1: FP32 links), 5 pair even + single odd,
                       // 6 tensor-core even + pair odd (binary16, one lattice, no clover)
  int big_lat = 0;     // index of the largest lattice of the problem (set before setup)
  bool one_lat = false;   // the problem has one lattice (set before setup)
  int kernels_per_iteration() const { return eo ? (SPR == PR64 ? 10 : 12) : (SPR == PR64 ? 7 : 8); }
  // streaming kernels: grid-stride with 8 blocks per SM per slot (few partial sums and atomic tickets);
  // stencil kernels: one block per tile (gy) so that the lattice is swept once in site order
  dim3 grid() const { return dim3(nslots, gyb); }
  dim3 grid_stencil() const { return dim3(nslots, gy); }
  // slots refilled together (the right-hand sides one thread carries must share a lattice)
  int group() const { return (eo && SPR != PR64) ? 2 : rpt; }   // pairs also for eo_kernel 1 (any choice)

  hp_status setup(int ns, int Vmax, const LatGeom* lats_dev, SlotState* st, const hp_solver_opts& o, double tol,
                  double delta, const LatGeom& gbig) {
    nslots = ns;
    memset(&a, 0, sizeof(a));
    a.lats = lats_dev;
    a.st = st;
    a.eo = eo ? 1 : 0;
    if (eo) Vmax = (Vmax + 1) / 2;   // every field lives on one parity
    a.Vmax = Vmax;
    gy = dslash_gridy(ctx, Vmax, NT, ns);
    gyb = std::max(1, std::min(gy, ctx->num_sms * 8));
    a.gy = gy;   // stride of the partial sums: the largest grid height of any kernel
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
    if (SPR != PR64) HP_TRY(alloc_field(ctx, "solve.rg", PR32, ns, Vmax, &a.rg));
    if (SPR == PR64) {
      HP_TRY(hp_ws(ctx, "solve.x", sizeof(double2) * 12 * (size_t)ns * Vmax, &p));
      a.x = (double2*)p;
      if (eo) {
        HP_TRY(hp_ws(ctx, "solve.xe", sizeof(double2) * 12 * (size_t)ns * Vmax, &p));
        a.xe = (double2*)p;
      }
    } else {   // float-float solution
      HP_TRY(alloc_field(ctx, "solve.xhi", PR32, ns, Vmax, &a.xff));
      FieldPtr lo;
      HP_TRY(alloc_field(ctx, "solve.xlo", PR32, ns, Vmax, &lo));
      a.xff.lo = lo.p;
      if (eo) {
        HP_TRY(alloc_field(ctx, "solve.xehi", PR32, ns, Vmax, &a.xeff));
        HP_TRY(alloc_field(ctx, "solve.xelo", PR32, ns, Vmax, &lo));
        a.xeff.lo = lo.p;
      }
    }
    if (eo) {
      HP_TRY(alloc_field(ctx, "solve.mid", SPR, ns, Vmax, &a.mid));
      if (SPR != PR64) HP_TRY(alloc_field(ctx, "solve.mid32", PR32, ns, Vmax, &a.mid32));
    }
    a.tol2 = tol * tol;
    a.delta2 = delta * delta;
    a.epsx2 = SPR == PR64 ? 0.0 : 1e-10;   // FP64 true residual after a 1e5 reduction
    a.maxiter = o.maxiter > 0 ? o.maxiter : 10000;
    // right-hand sides per thread of the stencil: fixed by the caller or autotuned on the largest lattice
    // stencil variant: fixed by the caller (right-hand sides per thread, 12-real links) or autotuned
    // on the largest lattice of the problem
    const int forced = o.rhs_per_thread % 100, full = (o.rhs_per_thread / 100) % 10 == 1,
              group = o.rhs_per_thread / 1000;
    if (forced == 1 || forced == 2 || forced == 4) {
      variant = 100 * group + 10 * forced + (full ? 1 : 0);
    } else if (eo) {
      // the full-lattice tuner cannot run on half-lattice fields: slot groups of 4 and 18-real links
      variant = 411;
    } else {
      k_w_fill<SPR><<<blocks_for(ctx, (long long)ns * Vmax, 256), 256, 0, ctx->stream>>>(a.p, Vmax, ns, 777ull);
      HP_LAUNCH_CHECK();
      HP_TRY(tune_rpt<SPR>(ctx, gbig, a.p, a.v, ns, Vmax, &variant));
    }
    rpt = variant_rpt(variant);
    if (eo) {   // the even-odd kernels take one right-hand side per thread; keep the group and link form
      variant = 100 * variant_group(variant) + 10 + (variant % 10);
      rpt = 1;
      if (SPR != PR64) {
        const int k = o.eo_kernel;
        if (k == 1 || k == 3 || k == 4 || k == 5 || k == 13 || k == 14 || (k == 6 && tc_ok())) eo_kernel = k;
        else HP_TRY(tune_eo(gbig));
      }
    }
    return HP_OK;
  }
  // ---- even-odd steps
  // grid of the even-odd kernels: one slot per block along x/z, tiles of NT sites along y
  dim3 eo_grid() const { return stencil_grid(variant, nslots, gy); }
  // masked launches that serve a few slots (exact and group steps, fresh starts): one block per
  // tile looping over the selected slots
  dim3 tile_grid() const { return dim3(1, gy, 1); }
  template <int REC, bool CL>
  hp_status eo_schur(int which) {   // which: 0 v = S p, 1 t = S s, 2 group update with e
    dim3 gr = eo_grid();
    constexpr int LPR = LinkPrecOf<SPR>::v;
    if constexpr (SPR != PR64) {   // two right-hand sides per thread, all slot pairs of a tile together
      if (which < 2 && eo_kernel >= 3) return eo_pair_v<CL>(which);
    }
    if (which == 0) {
      {
        ProfScope ps(ctx, "k_eo_even");
        k_eo_even<SPR, LPR, REC, SPR, NT, MASK_RUN, CL><<<gr, NT, 0, ctx->stream>>>(a, a.p, a.mid, nslots);
      }
      HP_LAUNCH_CHECK();
      ProfScope ps(ctx, SPR == PR64 ? "k_eo_odd_v<fp64>" : SPR == PR32 ? "k_eo_odd_v<fp32>" : SPR == PR16 ? "k_eo_odd_v<fp16>" : "k_eo_odd_v<bf16>");
      k_eo_odd<SPR, SPR, LPR, REC, NT, EPI_V, CL><<<gr, NT, 0, ctx->stream>>>(a, a.p, a.mid, a.v, nslots);
    } else if (which == 1) {
      {
        ProfScope ps(ctx, "k_eo_even");
        k_eo_even<SPR, LPR, REC, SPR, NT, MASK_RUN, CL><<<gr, NT, 0, ctx->stream>>>(a, a.s, a.mid, nslots);
      }
      HP_LAUNCH_CHECK();
      ProfScope ps(ctx, SPR == PR64 ? "k_eo_odd_t<fp64>" : SPR == PR32 ? "k_eo_odd_t<fp32>" : SPR == PR16 ? "k_eo_odd_t<fp16>" : "k_eo_odd_t<bf16>");
      k_eo_odd<SPR, SPR, LPR, REC, NT, EPI_T, CL><<<gr, NT, 0, ctx->stream>>>(a, a.s, a.mid, a.t, nslots);
    } else if (SPR != PR64) {
      {
        ProfScope ps(ctx, "k_eo_even<grp>");
        k_eo_even<EPR, PR32, 12, PR32, NT, MASK_GROUP, CL><<<tile_grid(), NT, 0, ctx->stream>>>(a, a.e, a.mid32, nslots);
      }
      HP_LAUNCH_CHECK();
      ProfScope ps(ctx, "k_eo_odd<grp>");
      k_eo_odd<EPR, PR32, PR32, 12, NT, EPI_G, CL><<<tile_grid(), NT, 0, ctx->stream>>>(a, a.e, a.mid32, a.rg, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // the V (which 0) or T (1) step with the pair kernels under a register budget of MINB blocks per SM,
  // links in LPR (binary16, or FP32: no conversions); the odd-site kernels sweep TPB tiles per block
  // (one partial-sum reduction per TPB tiles)
  template <int LPR, int MINB, bool CL>
  hp_status eo_pair(int which) {
    static_assert(SPR != PR64, "the pair kernels serve the FP32 / FP16 / BF16 iteration");
    constexpr int TPB = 2;
    const dim3 g2((nslots + 1) / 2, gy, 1), g2o((nslots + 1) / 2, (gy + TPB - 1) / TPB, 1);
    FieldPtr in = which == 0 ? a.p : a.s, out = which == 0 ? a.v : a.t;
    {
      ProfScope ps(ctx, "k_eo_even");
      k_eo2_even<SPR, LPR, NT, MINB, CL><<<g2, NT, 0, ctx->stream>>>(a, in, a.mid, nslots);
    }
    HP_LAUNCH_CHECK();
    if (which == 0) {
      ProfScope ps(ctx, SPR == PR32 ? "k_eo_odd_v<fp32>" : SPR == PR16 ? "k_eo_odd_v<fp16>" : "k_eo_odd_v<bf16>");
      k_eo2_odd<SPR, LPR, NT, MINB, EPI_V, CL, TPB><<<g2o, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    } else {
      ProfScope ps(ctx, SPR == PR32 ? "k_eo_odd_t<fp32>" : SPR == PR16 ? "k_eo_odd_t<fp16>" : "k_eo_odd_t<bf16>");
      k_eo2_odd<SPR, LPR, NT, MINB, EPI_T, CL, TPB><<<g2o, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // eo_kernel 5: the even-site pair kernel with the one-right-hand-side odd-site kernel
  template <bool CL>
  hp_status eo_mixed(int which) {
    constexpr int L16 = SPR == PR32 ? PR32 : PR16;
    const dim3 g2((nslots + 1) / 2, gy, 1), gr = eo_grid();
    FieldPtr in = which == 0 ? a.p : a.s, out = which == 0 ? a.v : a.t;
    {
      ProfScope ps(ctx, "k_eo_even");
      k_eo2_even<SPR, L16, NT, 4, CL><<<g2, NT, 0, ctx->stream>>>(a, in, a.mid, nslots);
    }
    HP_LAUNCH_CHECK();
    constexpr int LPR = LinkPrecOf<SPR>::v;
    if (which == 0) {
      ProfScope ps(ctx, SPR == PR32 ? "k_eo_odd_v<fp32>" : SPR == PR16 ? "k_eo_odd_v<fp16>" : "k_eo_odd_v<bf16>");
      k_eo_odd<SPR, SPR, LPR, 18, NT, EPI_V, CL><<<gr, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    } else {
      ProfScope ps(ctx, SPR == PR32 ? "k_eo_odd_t<fp32>" : SPR == PR16 ? "k_eo_odd_t<fp16>" : "k_eo_odd_t<bf16>");
      k_eo_odd<SPR, SPR, LPR, 18, NT, EPI_T, CL><<<gr, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // the tensor-core even-site kernel serves binary16 iterations of one lattice without the clover
  // term, up to 32 slots (four MMA row groups)
  bool tc_ok() const { return SPR == PR16 && !clover && one_lat && nslots <= 32; }
  // eo_kernel 6: the tensor-core even-site kernel with the odd-site pair kernel (4 resident blocks)
  template <bool CL>
  hp_status eo_tc(int which) {
    static_assert(SPR == PR16 && !CL, "binary16 without the clover term");
    constexpr int TPB = 2;
    const dim3 g2o((nslots + 1) / 2, (gy + TPB - 1) / TPB, 1);
    FieldPtr in = which == 0 ? a.p : a.s, out = which == 0 ? a.v : a.t;
    {
      ProfScope ps(ctx, "k_eo_even");
      const dim3 gt(ctx->num_sms * 4);
      switch ((nslots + 7) / 8) {
        case 1: k_eo3_even<1><<<gt, NT, 0, ctx->stream>>>(a, in, a.mid, nslots, big_lat); break;
        case 2: k_eo3_even<2><<<gt, NT, 0, ctx->stream>>>(a, in, a.mid, nslots, big_lat); break;
        case 3: k_eo3_even<3><<<gt, NT, 0, ctx->stream>>>(a, in, a.mid, nslots, big_lat); break;
        default: k_eo3_even<4><<<gt, NT, 0, ctx->stream>>>(a, in, a.mid, nslots, big_lat); break;
      }
    }
    HP_LAUNCH_CHECK();
    if (which == 0) {
      ProfScope ps(ctx, "k_eo_odd_v<fp16>");
      k_eo2_odd<SPR, PR16, NT, 4, EPI_V, CL, TPB><<<g2o, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    } else {
      ProfScope ps(ctx, "k_eo_odd_t<fp16>");
      k_eo2_odd<SPR, PR16, NT, 4, EPI_T, CL, TPB><<<g2o, NT, 0, ctx->stream>>>(a, in, a.mid, out, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  template <bool CL>
  hp_status eo_pair_v(int which) {   // eo_kernel = 10 L + B: B resident blocks, L = 1 FP32 links
    constexpr int L16 = SPR == PR32 ? PR32 : PR16;
    if constexpr (SPR == PR16 && !CL) {
      if (eo_kernel == 6 && tc_ok()) return eo_tc<CL>(which);
    }
    switch (eo_kernel) {
      case 5: return eo_mixed<CL>(which);
      case 3: return eo_pair<L16, 3, CL>(which);
      case 13: return eo_pair<PR32, 3, CL>(which);
      case 14: return eo_pair<PR32, 4, CL>(which);
      default: return eo_pair<L16, 4, CL>(which);
    }
  }
  // Autotuner of the even-odd iteration kernels: times the V step (k_eo_even + k_eo_odd) of every
  // variant -- one right-hand side per thread (1), the pair kernels at 3 or 4 resident blocks with
  // binary16 or FP32 links (3, 4, 13, 14), the even-site pair kernel with the one-right-hand-side
  // odd-site kernel (5) --
  // on this engine's fields with all slots marked running (a scratch copy of the slot states), and
  // keeps the fastest per (precision, lattice, slots).
  hp_status tune_eo(const LatGeom& gbig) {
    char key[160];
    snprintf(key, sizeof(key), "eo:%d:%d,%d,%d,%d:%d", SPR, gbig.L[0], gbig.L[1], gbig.L[2], gbig.L[3], nslots);
    auto it = ctx->autotune.find(key);
    if (it != ctx->autotune.end()) {
      eo_kernel = it->second;
      return HP_OK;
    }
    SlotState* keep = a.st;
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "solve.tune_state", sizeof(SlotState) * nslots, &p));
    std::vector<SlotState> st(nslots);
    memset(st.data(), 0, sizeof(SlotState) * nslots);
    for (auto& S : st) {   // every slot running on the largest lattice of the problem
      S.status = SLOT_RUN;
      S.lat = big_lat;
    }
    HP_CUDA(cudaMemcpyAsync(p, st.data(), sizeof(SlotState) * nslots, cudaMemcpyHostToDevice, ctx->stream));
    a.st = (SlotState*)p;
    cudaEvent_t e0, e1;
    HP_CUDA(cudaEventCreate(&e0));
    HP_CUDA(cudaEventCreate(&e1));
    float best = 1e30f;
    int choice = 4;
    const bool prof = ctx->profiling;
    ctx->profiling = false;
    hp_status status = HP_OK;
    for (int c : {1, 3, 4, 5, 13, 14}) {
      if (SPR == PR32 && c > 10) continue;   // FP32 iteration: FP32 links already
      eo_kernel = c;
      status = eo_step(0);
      if (status != HP_OK) break;
      cudaEventRecord(e0, ctx->stream);
      for (int i = 0; i < 3 && status == HP_OK; ++i) status = eo_step(0);
      cudaEventRecord(e1, ctx->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) {
        best = ms;
        choice = c;
      }
    }
    ctx->profiling = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    a.st = keep;
    HP_TRY(status);
    HP_CUDA(cudaMemsetAsync(a.cnt, 0, sizeof(unsigned int) * nslots, ctx->stream));
    eo_kernel = choice;
    ctx->autotune[key] = choice;
    return HP_OK;
  }
  hp_status eo_step(int which) {
    const bool full = variant_rec(variant) == 18 && SPR != PR64;
    if (clover) return full ? eo_schur<18, true>(which) : eo_schur<12, true>(which);
    return full ? eo_schur<18, false>(which) : eo_schur<12, false>(which);
  }
  hp_status eo_exact() {
    dim3 gr = eo_grid();
    {
      ProfScope ps(ctx, PX == PR64 ? "k_eo_x1<fp64>" : "k_eo_x1<ff>");
      k_eo_x1<PX, NT><<<tile_grid(), NT, 0, ctx->stream>>>(a, nslots);
    }
    HP_LAUNCH_CHECK();
    {
      ProfScope ps(ctx, PX == PR64 ? "k_eo_x2<fp64>" : "k_eo_x2<ff>");
      k_eo_x2<SPR, PX, NT><<<tile_grid(), NT, 0, ctx->stream>>>(a, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  template <int RPT, int REC, bool CL>
  hp_status stencil_steps_rpt(int which) {
    dim3 gr = stencil_grid(variant, nslots, gy);
    if (which == 0) {
      ProfScope ps(ctx, SPR == PR64 ? "k_bicg_v<fp64>" : SPR == PR32 ? "k_bicg_v<fp32>" : SPR == PR16 ? "k_bicg_v<fp16>" : "k_bicg_v<bf16>");
      k_wds<SPR, RPT, NT, EPI_V, REC, CL><<<gr, NT, 0, ctx->stream>>>(a, a.p, a.v, nslots);
    } else {
      ProfScope ps(ctx, SPR == PR64 ? "k_bicg_t<fp64>" : SPR == PR32 ? "k_bicg_t<fp32>" : SPR == PR16 ? "k_bicg_t<fp16>" : "k_bicg_t<bf16>");
      k_wds<SPR, RPT, NT, EPI_T, REC, CL><<<gr, NT, 0, ctx->stream>>>(a, a.s, a.t, nslots);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  template <bool CL>
  hp_status stencil_step_cl(int which) {
    const bool full = variant_rec(variant) == 18 && SPR != PR64;
    if (rpt == 4) return full ? stencil_steps_rpt<4, 18, CL>(which) : stencil_steps_rpt<4, 12, CL>(which);
    if (rpt == 2) return full ? stencil_steps_rpt<2, 18, CL>(which) : stencil_steps_rpt<2, 12, CL>(which);
    return full ? stencil_steps_rpt<1, 18, CL>(which) : stencil_steps_rpt<1, 12, CL>(which);
  }
  hp_status stencil_step(int which) { return clover ? stencil_step_cl<true>(which) : stencil_step_cl<false>(which); }
  hp_status init() {
    if (eo) {
      {
        ProfScope ps(ctx, "k_eo_init");
        k_eo_init<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a, nslots);
      }
      HP_LAUNCH_CHECK();
      if (SPR != PR64) {
        const dim3 gr = eo_grid();
        {
          ProfScope ps(ctx, "k_eo_src");
          k_eo_src<NT><<<tile_grid(), NT, 0, ctx->stream>>>(a, nslots);
        }
        HP_LAUNCH_CHECK();
        {
          ProfScope ps(ctx, "k_eo_r0");
          k_eo_r0<SPR, NT><<<tile_grid(), NT, 0, ctx->stream>>>(a, nslots);
        }
        HP_LAUNCH_CHECK();
      }
      // FP64: x_e = d_e^-1 b_e and the initial residual of the Schur system; mixed: only slots
      // whose FP32 start residual is already at the tolerance
      return eo_exact();
    }
    {
      ProfScope ps(ctx, "k_bicg_init");
      k_bicg_init<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status iteration() {
    if (eo) {
      HP_TRY(eo_step(0));
      { ProfScope ps(ctx, "k_bicg_s"); k_bicg_s<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
      HP_TRY(eo_step(1));
      { ProfScope ps(ctx, "k_bicg_xr"); k_bicg_xr<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
      if (SPR != PR64) HP_TRY(eo_step(2));
      { ProfScope ps(ctx, "k_ru_accum"); k_ru_accum<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
      HP_TRY(eo_exact());
      { ProfScope ps(ctx, "k_bicg_p"); k_bicg_p<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
      HP_LAUNCH_CHECK();
      return HP_OK;
    }
    HP_TRY(stencil_step(0));
    { ProfScope ps(ctx, "k_bicg_s"); k_bicg_s<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    HP_TRY(stencil_step(1));
    { ProfScope ps(ctx, "k_bicg_xr"); k_bicg_xr<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    if (SPR != PR64) {
      ProfScope ps(ctx, "k_grp_update");
      k_grp_update<SPR, EPR, NT><<<grid_stencil(), NT, 0, ctx->stream>>>(a);
    }
    { ProfScope ps(ctx, "k_ru_accum"); k_ru_accum<SPR, EPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    {
      ProfScope ps(ctx, SPR == PR64 ? "k_ru_residual<fp64>" : "k_ru_residual<ff>");
      k_ru_residual<SPR, NT><<<grid_stencil(), NT, 0, ctx->stream>>>(a);
    }
    { ProfScope ps(ctx, "k_bicg_p"); k_bicg_p<SPR, NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // copy the solutions of the harvested slots that the caller keeps (lattice 0, first n_keep right-hand sides)
  hp_status keep(const std::vector<int>& done_slots, const std::vector<SlotState>& host, const SolveProblem& pb) {
    std::vector<int> list;
    for (int sl : done_slots) {
      const SlotState& S = host[sl];
      const int64_t j = (int64_t)(S.m - pb.first[0]) * 12 + S.a;
      if (S.lat == 0 && j < pb.n_keep) list.push_back(sl);
    }
    const int n = (int)list.size();
    if (!n) return HP_OK;
    for (int i = 0; i < n; ++i) {
      const SlotState& S = host[list[i]];
      list.push_back((int)((int64_t)(S.m - pb.first[0]) * 12 + S.a));
    }
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "solve.keep", sizeof(int) * 2 * (size_t)nslots, &p));
    int* d = (int*)p;
    HP_CUDA(cudaMemcpyAsync(d, list.data(), sizeof(int) * 2 * n, cudaMemcpyHostToDevice, ctx->stream));
    {
      ProfScope ps(ctx, "k_w_keep");
      k_w_keep<<<blocks_for(ctx, (long long)n * pb.lats[0].V, 256), 256, 0, ctx->stream>>>(a, d, d + n, n, pb.x_keep,
                                                                                        pb.lats[0]);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status harvest(const std::vector<int>& done_slots, const SolveProblem& pb, int* dev_slots) {
    if (eo) {
      {
        ProfScope ps(ctx, "k_quad");
        k_eo_quad<NT><<<grid(), NT, 0, ctx->stream>>>(a, nslots);
      }
      HP_LAUNCH_CHECK();
      if (pb.want_grad && !done_slots.empty()) {
        HP_CUDA(cudaMemcpyAsync(dev_slots, done_slots.data(), sizeof(int) * done_slots.size(),
                                cudaMemcpyHostToDevice, ctx->stream));
        for (size_t L = 0; L < pb.lats.size(); ++L) {
          ProfScope ps(ctx, "k_w_grad");
          k_eo_grad<<<blocks_for(ctx, pb.lats[L].V, 256), 256, 0, ctx->stream>>>(a, (int)L, dev_slots,
                                                                                  (int)done_slots.size(),
                                                                                  pb.grad_dev[L], pb.lats[L]);
        }
        HP_LAUNCH_CHECK();
      }
      return HP_OK;
    }
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

template <int SPR, int RPT, int REC>
static hp_status launch_dslash_rpt(hp_ctx* ctx, const WArgs& a, FieldPtr in, FieldPtr out, int nrhs, int V,
                                   int variant, bool clover) {
  constexpr int NT = 128;
  dim3 grid = stencil_grid(variant, nrhs, dslash_gridy(ctx, V, NT, nrhs));
  {
    ProfScope ps(ctx, SPR == PR64 ? "k_wds<fp64>" : SPR == PR32 ? "k_wds<fp32>" : SPR == PR16 ? "k_wds<fp16>" : "k_wds<bf16>");
    if (clover)
      k_wds<SPR, RPT, NT, EPI_PLAIN, REC, true><<<grid, NT, 0, ctx->stream>>>(a, in, out, nrhs);
    else
      k_wds<SPR, RPT, NT, EPI_PLAIN, REC, false><<<grid, NT, 0, ctx->stream>>>(a, in, out, nrhs);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}


// out = D in for nrhs fields of one lattice, in the given variant
template <int SPR>
static hp_status launch_dslash(hp_ctx* ctx, const LatGeom& g, FieldPtr in, FieldPtr out, int nrhs, int Vmax,
                               int variant) {
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "dslash.lat", sizeof(LatGeom), &p));
  HP_CUDA(cudaMemcpyAsync(p, &g, sizeof(LatGeom), cudaMemcpyHostToDevice, ctx->stream));
  WArgs a;
  memset(&a, 0, sizeof(a));
  a.lats = (const LatGeom*)p;
  a.Vmax = Vmax;
  const bool full = variant_rec(variant) == 18 && SPR != PR64;
  switch (variant_rpt(variant)) {
    case 1: return full ? launch_dslash_rpt<SPR, 1, 18>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0) : launch_dslash_rpt<SPR, 1, 12>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0);
    case 2: return full ? launch_dslash_rpt<SPR, 2, 18>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0) : launch_dslash_rpt<SPR, 2, 12>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0);
    default: return full ? launch_dslash_rpt<SPR, 4, 18>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0) : launch_dslash_rpt<SPR, 4, 12>(ctx, a, in, out, nrhs, g.V, variant, g.clover != 0);
  }
}

// apply: the variant follows nrhs so that parity tests reach every kernel: nrhs 1-2 -> 1 per thread,
// 3-4 -> 2, >= 5 -> 4; odd nrhs with 12-real links, even with 18-real links
static int apply_variant(int nrhs) { return 10 * (nrhs >= 5 ? 4 : (nrhs >= 3 ? 2 : 1)) + (nrhs % 2 ? 0 : 1); }

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
  HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V, apply_variant(nrhs)));
  k_w_to_canonical<SPR><<<blocks_for(ctx, (long long)nrhs * V, 256), 256, 0, ctx->stream>>>(fo, V, nrhs, (double2*)dout);
  HP_LAUNCH_CHECK();
  if (out_host) {
    HP_CUDA(cudaMemcpyAsync(out, dout, cbytes, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return HP_OK;
}

// ================================================================ Schur-complement apply
// canonical complex [nrhs][V][12] -> half-lattice field of parity `par` (slot = right-hand side)
template <int SPR>
__global__ void k_eo_from_canonical(const double2* __restrict__ in, FieldPtr f, LatGeom g, int Vmax, int nrhs,
                                    int par) {
  const int Vh = g.V >> 1;
  const long long total = (long long)nrhs * Vh;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(t / Vh), h = (int)(t - (long long)slot * Vh);
    int x[4], st[4];
    const int site = eo_site(g, h, par, x, st);
    typedef typename Real_of<SPR>::T R;
    cplx<R> s[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
      const double2 v = in[((size_t)slot * g.V + site) * 12 + k];
      s[k] = {(R)v.x, (R)v.y};
    }
    SpinorIO<SPR>::store(f, Vmax, slot, h, s);
  }
}

// half-lattice field of parity `par` -> canonical complex [nrhs][V][12], zero on the other parity
template <int SPR>
__global__ void k_eo_to_canonical(FieldPtr f, LatGeom g, int Vmax, int nrhs, int par, double2* __restrict__ out) {
  const long long total = (long long)nrhs * g.V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(t / g.V), site = (int)(t - (long long)slot * g.V);
    double2* o = out + ((size_t)slot * g.V + site) * 12;
    if (site_parity(g, site) != par) {
#pragma unroll
      for (int k = 0; k < 12; ++k) o[k] = make_double2(0.0, 0.0);
      continue;
    }
    typedef typename Real_of<SPR>::T R;
    cplx<R> s[12];
    SpinorIO<SPR>::load(f, Vmax, slot, site >> 1, s);
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = make_double2((double)s[k].x, (double)s[k].y);
  }
}

// out = S in on the odd sites, S = A_o - kappa^2 H_oe A_e^-1 H_eo (the even-odd iteration's operator),
// through the solver's own launches: a WilsonEngine set up for the right-hand sides as running slots
// of one lattice, its V step v = S p, in the iteration precision SPR
template <int SPR>
static hp_status schur_apply_t(hp_ctx* ctx, const LatGeom& g, int nrhs, int eo_kernel, const double* in,
                               double* out) {
  WilsonEngine<SPR> e{ctx};
  e.eo = true;
  e.clover = g.clover != 0;
  e.one_lat = true;
  const int ns = (nrhs + WilsonEngine<SPR>::GROUP_MAX - 1) / WilsonEngine<SPR>::GROUP_MAX * WilsonEngine<SPR>::GROUP_MAX;
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "schur.lat", sizeof(LatGeom), &p));
  LatGeom* lat_dev = (LatGeom*)p;
  HP_CUDA(cudaMemcpyAsync(lat_dev, &g, sizeof(LatGeom), cudaMemcpyHostToDevice, ctx->stream));
  HP_TRY(hp_ws(ctx, "schur.state", sizeof(SlotState) * ns, &p));
  SlotState* st_dev = (SlotState*)p;
  std::vector<SlotState> st(ns);
  memset(st.data(), 0, sizeof(SlotState) * ns);
  for (int i = 0; i < nrhs; ++i) st[i].status = SLOT_RUN;
  HP_CUDA(cudaMemcpyAsync(st_dev, st.data(), sizeof(SlotState) * ns, cudaMemcpyHostToDevice, ctx->stream));
  hp_solver_opts o;
  memset(&o, 0, sizeof(o));
  o.eo_kernel = eo_kernel;
  HP_TRY(e.setup(ns, g.V, lat_dev, st_dev, o, 1e-10, 0.0, g));
  size_t nb = 0;
  const size_t fb = field_bytes(SPR, ns, e.a.Vmax, &nb);
  HP_CUDA(cudaMemsetAsync(e.a.rh.p, 0, fb, ctx->stream));   // the V step's epilogue reads r^
  if (nb) HP_CUDA(cudaMemsetAsync(e.a.rh.nrm, 0, nb, ctx->stream));
  const size_t cbytes = sizeof(double2) * 12 * (size_t)nrhs * g.V;
  const void* din = nullptr;
  HP_TRY(hp_device_view(ctx, in, cbytes, "schur.canon_in", &din));
  double* dout = out;
  const bool out_host = !hp_is_device_ptr(out);
  if (out_host) {
    HP_TRY(hp_ws(ctx, "schur.canon_out", cbytes, &p));
    dout = (double*)p;
  }
  const long long nh = (long long)nrhs * (g.V >> 1);
  k_eo_from_canonical<SPR><<<blocks_for(ctx, nh, 256), 256, 0, ctx->stream>>>((const double2*)din, e.a.p, g,
                                                                               e.a.Vmax, nrhs, 1);
  HP_LAUNCH_CHECK();
  HP_TRY(e.eo_step(0));
  k_eo_to_canonical<SPR><<<blocks_for(ctx, (long long)nrhs * g.V, 256), 256, 0, ctx->stream>>>(
      e.a.v, g, e.a.Vmax, nrhs, 1, (double2*)dout);
  HP_LAUNCH_CHECK();
  if (out_host) HP_CUDA(cudaMemcpyAsync(out, dout, cbytes, cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
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

// Autotuner: times the stencil with 1, 2 and 4 right-hand sides per thread on
// the given fields (3 launches each, CUDA events) and caches the fastest per
// (lattice, precision, number of right-hand sides).
template <int SPR>
static hp_status tune_rpt(hp_ctx* ctx, const LatGeom& g, FieldPtr fi, FieldPtr fo, int nrhs, int Vmax, int* best) {
  char key[160];
  snprintf(key, sizeof(key), "wds:%d:%d,%d,%d,%d:%d", SPR, g.L[0], g.L[1], g.L[2], g.L[3], nrhs);
  auto it = ctx->autotune.find(key);
  if (it != ctx->autotune.end()) {
    *best = it->second;
    return HP_OK;
  }
  cudaEvent_t e0, e1;
  HP_CUDA(cudaEventCreate(&e0));
  HP_CUDA(cudaEventCreate(&e1));
  float best_ms = 1e30f;
  int best_r = 10;
  const int cands[14] = {10, 11, 20, 21, 40, 41, 410, 411, 421, 810, 811, 821, 1611, 1621};
  for (int c : cands) {
    if (variant_rpt(c) > 1 && variant_rpt(c) > nrhs) continue;
    if (SPR == PR64 && (variant_rec(c) == 18 || variant_rpt(c) > 1)) continue;
    if (variant_group(c) > 0 && variant_group(c) >= nrhs) continue;
    HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, Vmax, c));
    HP_CUDA(cudaEventRecord(e0, ctx->stream));
    for (int i = 0; i < 3; ++i) HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, Vmax, c));
    HP_CUDA(cudaEventRecord(e1, ctx->stream));
    HP_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    HP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (ms < best_ms) {
      best_ms = ms;
      best_r = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->autotune[key] = best_r;
  *best = best_r;
  return HP_OK;
}

template <int SPR>
static hp_status bench_wilson_t(hp_ctx* ctx, const LatGeom& g, int nrhs, int iters, double* ms) {
  const int V = g.V;
  FieldPtr fi, fo;
  HP_TRY(alloc_field(ctx, "bench.in", SPR, nrhs, V, &fi));
  HP_TRY(alloc_field(ctx, "bench.out", SPR, nrhs, V, &fo));
  k_w_fill<SPR><<<blocks_for(ctx, (long long)nrhs * V, 256), 256, 0, ctx->stream>>>(fi, V, nrhs, 12345ull);
  HP_LAUNCH_CHECK();
  int rpt = 1;
  HP_TRY(tune_rpt<SPR>(ctx, g, fi, fo, nrhs, V, &rpt));
  for (int w = 0; w < 3; ++w) HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V, rpt));
  cudaEvent_t a, b;
  HP_CUDA(cudaEventCreate(&a));
  HP_CUDA(cudaEventCreate(&b));
  HP_CUDA(cudaEventRecord(a, ctx->stream));
  for (int i = 0; i < iters; ++i) HP_TRY(launch_dslash<SPR>(ctx, g, fi, fo, nrhs, V, rpt));
  HP_CUDA(cudaEventRecord(b, ctx->stream));
  HP_CUDA(cudaEventSynchronize(b));
  float t = 0.f;
  HP_CUDA(cudaEventElapsedTime(&t, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *ms = (double)t / iters;
  return HP_OK;
}

// generic slot scheduler shared by both operator families
#include "hp_schedule.cuh"

// generic slot scheduler shared by both operator families
#include "hp_schedule.cuh"

// the per-precision entry points (one translation unit each)
template <int SPR>
hp_status wilson_apply_prec(hp_ctx* ctx, const LatGeom& g, int nrhs, const double* in, double* out) {
  return apply_wilson_t<SPR>(ctx, g, nrhs, in, out);
}
template <int SPR>
hp_status wilson_schur_prec(hp_ctx* ctx, const LatGeom& g, int nrhs, int eo_kernel, const double* in, double* out) {
  return schur_apply_t<SPR>(ctx, g, nrhs, eo_kernel, in, out);
}
template <int SPR>
hp_status wilson_bench_prec(hp_ctx* ctx, const LatGeom& g, int nrhs, int iters, double* ms) {
  return bench_wilson_t<SPR>(ctx, g, nrhs, iters, ms);
}
template <int SPR>
hp_status wilson_solve_prec(hp_ctx* ctx, SolveProblem& pb, SolveResult& res, bool eo, bool clover, double delta) {
  WilsonEngine<SPR> e{ctx};
  e.eo = eo;
  e.clover = clover;
  return run_schedule(ctx, e, pb, res, 12, delta);
}

#define HP_WILSON_INSTANTIATE(SPR, SUFFIX)                                                                  \
  hp_status hp_wilson_apply_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, const double* in, double* out) { \
    return wilson_apply_prec<SPR>(ctx, g, nrhs, in, out);                                                     \
  }                                                                                                           \
  hp_status hp_wilson_bench_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, int iters, double* ms) {        \
    return wilson_bench_prec<SPR>(ctx, g, nrhs, iters, ms);                                                   \
  }                                                                                                           \
  hp_status hp_wilson_schur_##SUFFIX(hp_ctx* ctx, const LatGeom& g, int nrhs, int eo_kernel, const double* in,  \
                                      double* out) {                                                          \
    return wilson_schur_prec<SPR>(ctx, g, nrhs, eo_kernel, in, out);                                          \
  }                                                                                                           \
  hp_status hp_wilson_solve_##SUFFIX(hp_ctx* ctx, SolveProblem& pb, SolveResult& res, bool eo, bool clover,   \
                                     double delta) {                                                          \
    return wilson_solve_prec<SPR>(ctx, pb, res, eo, clover, delta);                                          \
  }
