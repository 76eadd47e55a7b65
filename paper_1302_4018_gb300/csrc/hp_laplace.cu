// Shifted periodic Laplacian (the control problem of Section 5):
//   (A x)(s) = (8 + m + mu(s)) x(s) - sum_mu [x(s + mu) + x(s - mu)]
// in FP64, and multi-right-hand-side CG for the quadratures v^H A^-1 v.
// A is real, so a complex probe is solved as two real right-hand sides
// (its real and imaginary parts); the cross terms of v^H x cancel because
// A is symmetric.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "hp_internal.h"

static int lblocks(hp_ctx* ctx, long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)ctx->num_sms * 16;
  return (int)std::max(1LL, std::min(b, cap));
}

__device__ __forceinline__ double lap_site(const LatGeom& g, const double* __restrict__ x, int site) {
  if (g.csr_rp) {   // a general sparse matrix: row `site` of A times x
    double acc = 0.0;
    for (int e = g.csr_rp[site]; e < g.csr_rp[site + 1]; ++e) acc += g.csr_val[e] * __ldg(x + g.csr_ci[e]);
    return acc;
  }
  int r = site, st = 1;
  double acc = 0.0;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int L = g.L[j];
    const int xj = r % L;
    r /= L;
    const int fw = (xj + 1 == L) ? site - (L - 1) * st : site + st;
    const int bw = (xj == 0) ? site + (L - 1) * st : site - st;
    acc += __ldg(x + fw) + __ldg(x + bw);
    st *= L;
  }
  const double diag = 8.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0);
  return diag * __ldg(x + site) - acc;
}

__global__ void k_lap_apply(LatGeom g, const double* __restrict__ in, double* __restrict__ out, int nrhs) {
  const long long total = (long long)nrhs * g.V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    int rhs = (int)(t / g.V), site = (int)(t - (long long)rhs * g.V);
    out[t] = lap_site(g, in + (size_t)rhs * g.V, site);
  }
}

hp_status hp_apply_laplace(hp_ctx* ctx, LatGeom g, int nrhs, const double* in, double* out) {
  const size_t bytes = sizeof(double) * (size_t)nrhs * g.V;
  const void* din = nullptr;
  HP_TRY(hp_device_view(ctx, in, bytes, "apply.lap_in", &din));
  double* dout = out;
  bool out_host = !hp_is_device_ptr(out);
  if (out_host) {
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "apply.lap_out", bytes, &p));
    dout = (double*)p;
  }
  {
    ProfScope ps(ctx, "k_lap_apply");
    k_lap_apply<<<lblocks(ctx, (long long)nrhs * g.V, 256), 256, 0, ctx->stream>>>(g, (const double*)din, dout, nrhs);
  }
  HP_LAUNCH_CHECK();
  if (out_host) {
    HP_CUDA(cudaMemcpyAsync(out, dout, bytes, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return HP_OK;
}

// ------------------------------------------------------------------ CG kernels
struct LArgs {
  const LatGeom* lats;
  SlotState* st;
  double* part;
  unsigned int* cnt;
  int Vmax, gy;
  double *x, *r, *p, *q;   // [slot][Vmax]
  double tol2;
  int maxiter;
  int by_slot;   // 1: grid (tiles, slots), 0: grid (slots, tiles)
};

#define LSLOT(COND)                                                \
  const int slot = a.by_slot ? blockIdx.y : blockIdx.x;            \
  const int bx = a.by_slot ? blockIdx.x : blockIdx.y;              \
  const int gx = a.by_slot ? gridDim.x : gridDim.y;                \
  SlotState* S = a.st + slot;                                      \
  if (!(COND)) return;                                             \
  const LatGeom g = a.lats[S->lat];                                \
  const int ntiles = (g.V + NT - 1) / NT;                          \
  if (bx >= ntiles) return;                                        \
  const int nparts = min(gx, ntiles);                              \
  double* part = a.part + (size_t)slot * 4 * a.gy;                 \
  const size_t off = (size_t)slot * a.Vmax;                        \
  (void)nparts;                                                    \
  (void)part;

__device__ __forceinline__ double lap_source(const LatGeom& g, int site, int m, int part) {
  double2 v = g.ptab[probe_phase(g, (uint32_t)site, (uint32_t)m)];
  return part == 0 ? v.x : v.y;
}

template <int NQ, int NT>
__device__ __forceinline__ void lreduce(double (&v)[NQ], double* part, int gy, int bx) {
  __shared__ double sh[NQ][NT / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int qq = 0; qq < NQ; ++qq) {
    double t = v[qq];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[qq][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int qq = 0; qq < NQ; ++qq) {
      double t = 0.0;
      for (int w = 0; w < NT / 32; ++w) t += sh[qq][w];
      part[(size_t)qq * gy + bx] = t;
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_cg_init(LArgs a) {
  LSLOT(S->status == SLOT_INIT)
  double acc[1] = {0.0};
  const int m = S->m, pa = S->a;
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double b = lap_source(g, site, m, pa);
    a.x[off + site] = 0.0;
    a.r[off + site] = b;
    a.p[off + site] = b;
    acc[0] += b * b;
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->bnorm2 = tot[0];
      S->rnorm2 = tot[0];
      S->rmax2 = tot[0];
      S->rho = make_double2(tot[0], 0.0);
      S->iters = 0;
      S->updates = 0;
      S->need_update = 0;
      S->restart = 0;
      S->true_res2 = tot[0];
      S->gauss = 0.0;
      S->radau = g.quad_mu > 0.0 ? 1.0 / g.quad_mu : 0.0;
      S->status = tot[0] > 0.0 ? SLOT_RUN : SLOT_DONE;
      a.cnt[slot] = 0;
    }
  }
}

// q = A p ; alpha = rr / (p, q)
template <int NT>
__global__ void __launch_bounds__(NT) k_cg_ap(LArgs a) {
  LSLOT(S->status == SLOT_RUN)
  double acc[1] = {0.0};
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double qv = lap_site(g, a.p + off, site);
    a.q[off + site] = qv;
    acc[0] += a.p[off + site] * qv;
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->alpha = make_double2(tot[0] != 0.0 ? S->rho.x / tot[0] : 0.0, 0.0);
      S->gauss += S->alpha.x * S->rho.x;   // Gauss rule: G_{k+1} = G_k + gamma_k ||r_k||^2
      S->restart = 0;
      S->sloppy_mv += 1;
      a.cnt[slot] = 0;
    }
  }
}

// x += alpha p ; r -= alpha q ; beta = rr' / rr
template <int NT>
__global__ void __launch_bounds__(NT) k_cg_xr(LArgs a) {
  LSLOT(S->status == SLOT_RUN)
  const double al = S->alpha.x;
  double acc[1] = {0.0};
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    a.x[off + site] += al * a.p[off + site];
    double rv = a.r[off + site] - al * a.q[off + site];
    a.r[off + site] = rv;
    acc[0] += rv * rv;
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      const double rr = tot[0];
      const double delta = S->rho.x != 0.0 ? rr / S->rho.x : 0.0;
      S->beta = make_double2(delta, 0.0);
      S->rho = make_double2(rr, 0.0);
      S->rnorm2 = rr;
      S->iters += 1;
      if (g.quad_mu > 0.0) {   // Gauss-Radau: gt_{k+1} = (gt_k - gamma_k) / (mu (gt_k - gamma_k) + delta_{k+1})
        const double d = S->radau - S->alpha.x;
        const double den = g.quad_mu * d + delta;
        S->radau = den > 0.0 ? fmax(d, 0.0) / den : 0.0;
      }
      if (S->iters >= a.maxiter) {
        S->status = SLOT_FAIL;
        S->need_update = 1;
      } else if (g.quad_tol > 0.0) {   // stop on the quadrature bracket: no residual test, no restart
        if (S->radau * rr <= g.quad_tol * S->gauss || rr == 0.0 || !(rr == rr)) {
          S->true_res2 = rr;
          S->status = (rr == rr) ? SLOT_DONE : SLOT_FAIL;
        }
      } else if (rr <= a.tol2 * S->bnorm2 || !(rr == rr)) {
        S->need_update = 1;
      }
      a.cnt[slot] = 0;
    }
  }
}

// true residual r = b - A x
template <int NT>
__global__ void __launch_bounds__(NT) k_cg_true(LArgs a) {
  LSLOT(S->need_update)
  double acc[1] = {0.0};
  const int m = S->m, pa = S->a;
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    double rv = lap_source(g, site, m, pa) - lap_site(g, a.x + off, site);
    a.r[off + site] = rv;
    acc[0] += rv * rv;
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      const double rr = tot[0];
      S->true_res2 = rr;
      S->updates += 1;
      S->fp64_mv += 1;
      S->need_update = 0;
      if (S->status == SLOT_RUN) {
        if (rr <= a.tol2 * S->bnorm2) {
          S->status = SLOT_DONE;
        } else {   // continue from the true residual with p = r
          S->rho = make_double2(rr, 0.0);
          S->rnorm2 = rr;
          S->restart = 1;
        }
      }
      a.cnt[slot] = 0;
    }
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_cg_p(LArgs a) {
  LSLOT(S->status == SLOT_RUN)
  const double be = S->restart ? 0.0 : S->beta.x;
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    a.p[off + site] = a.r[off + site] + be * a.p[off + site];
  }
}

template <int NT>
__global__ void __launch_bounds__(NT) k_lquad(LArgs a) {
  LSLOT(S->status == SLOT_DONE || S->status == SLOT_FAIL)
  double acc[1] = {0.0};
  const int m = S->m, pa = S->a;
  for (int tile = bx; tile < ntiles; tile += gx) {
    const int site = tile * NT + threadIdx.x;
    if (site >= g.V) continue;
    acc[0] += lap_source(g, site, m, pa) * a.x[off + site];
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      S->q = make_double2(tot[0], 0.0);
      a.cnt[slot] = 0;
    }
  }
}

// g(site) += x(site)^2 over harvested slots of one lattice (A real symmetric: A^-H v = x)
__global__ void k_lgrad(LArgs a, int lat, const int* __restrict__ slots, int nsl, double* __restrict__ grad, int V) {
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < V; site += gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int i = 0; i < nsl; ++i) {
      const int slot = slots[i];
      if (a.st[slot].lat != lat) continue;
      double xv = a.x[(size_t)slot * a.Vmax + site];
      acc += xv * xv;
    }
    grad[site] += acc;
  }
}

struct LaplaceEngine {
  static constexpr int NT = 256;
  int kernels_per_iteration() const { return 4; }
  static constexpr int GROUP_MAX = 1;
  hp_ctx* ctx;
  LArgs a;
  int nslots, gy;
  // A sparse matrix runs with slots along y: the blocks of one slot are scheduled together,
  // so the vector its rows gather from stays in L2 while the slot runs (slots along x would
  // interleave all of them, and every gather of a renumbered matrix would be a DRAM sector).
  // The lattice stencil reads neighbours that are near in memory; there slots along x measured
  // faster (all slots stream at once).
  dim3 grid() const { return a.by_slot ? dim3(gy, nslots) : dim3(nslots, gy); }
  int group() const { return 1; }
  hp_status setup(int ns, int Vmax, const LatGeom* lats_dev, SlotState* st, const hp_solver_opts& o, double tol,
                  double, const LatGeom& big) {
    nslots = ns;
    memset(&a, 0, sizeof(a));
    a.lats = lats_dev;
    a.st = st;
    a.Vmax = Vmax;
    int ntiles = (Vmax + NT - 1) / NT;
    gy = std::max(1, std::min(std::min(ntiles, ctx->num_sms * 4), 65535));
    a.gy = gy;
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "solve.part", sizeof(double) * 4 * (size_t)ns * gy, &p));
    a.part = (double*)p;
    HP_TRY(hp_ws(ctx, "solve.cnt", sizeof(unsigned int) * ns, &p));
    a.cnt = (unsigned int*)p;
    HP_CUDA(cudaMemsetAsync(a.cnt, 0, sizeof(unsigned int) * ns, ctx->stream));
    const size_t fb = sizeof(double) * (size_t)ns * Vmax;
    HP_TRY(hp_ws(ctx, "solve.lx", fb, &p));
    a.x = (double*)p;
    HP_TRY(hp_ws(ctx, "solve.lr", fb, &p));
    a.r = (double*)p;
    HP_TRY(hp_ws(ctx, "solve.lp", fb, &p));
    a.p = (double*)p;
    HP_TRY(hp_ws(ctx, "solve.lq", fb, &p));
    a.q = (double*)p;
    a.tol2 = tol * tol;
    a.maxiter = o.maxiter > 0 ? o.maxiter : 10000;
    a.by_slot = big.csr_rp != nullptr;
    return HP_OK;
  }
  hp_status init() {
    {
      ProfScope ps(ctx, "k_cg_init");
      k_cg_init<NT><<<grid(), NT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status iteration() {
    { ProfScope ps(ctx, "k_cg_ap"); k_cg_ap<NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_cg_xr"); k_cg_xr<NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_cg_true"); k_cg_true<NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_cg_p"); k_cg_p<NT><<<grid(), NT, 0, ctx->stream>>>(a); }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status harvest(const std::vector<int>& done_slots, const SolveProblem& pb, int* dev_slots) {
    {
      ProfScope ps(ctx, "k_lquad");
      k_lquad<NT><<<grid(), NT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    if (pb.want_grad && !done_slots.empty()) {
      HP_CUDA(cudaMemcpyAsync(dev_slots, done_slots.data(), sizeof(int) * done_slots.size(), cudaMemcpyHostToDevice,
                              ctx->stream));
      for (size_t L = 0; L < pb.lats.size(); ++L) {
        ProfScope ps(ctx, "k_lgrad");
        k_lgrad<<<lblocks(ctx, pb.lats[L].V, 256), 256, 0, ctx->stream>>>(a, (int)L, dev_slots, (int)done_slots.size(),
                                                                          pb.grad_dev[L], pb.lats[L].V);
      }
      HP_LAUNCH_CHECK();
    }
    return HP_OK;
  }
};

#include "hp_schedule.cuh"

hp_status hp_solve_laplace(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  LaplaceEngine e{ctx};
  return run_schedule(ctx, e, pb, res, 12, 0.0);
}
