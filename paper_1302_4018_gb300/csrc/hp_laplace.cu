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
  double* dc;    // deflation: V^T b of each slot's source, [slot][defl_k]
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

// the solved source: the probe, projected off the deflated eigenvectors when there are any
__device__ __forceinline__ double lap_src(const LatGeom& g, const LArgs& a, int slot, int site, int m, int part) {
  double b = lap_source(g, site, m, part);
  if (g.defl_k) {
    const double* c = a.dc + (size_t)slot * g.defl_k;
    for (int j = 0; j < g.defl_k; ++j) b -= c[j] * g.defl_V[(size_t)j * g.V + site];
  }
  return b;
}

// deflation coefficients c_j = V_j^T b of the slots being filled: block (j, slot), one sum over
// the lattice in a fixed order
template <int NT>
__global__ void __launch_bounds__(NT) k_cg_defl(LArgs a) {
  const int j = blockIdx.x, slot = blockIdx.y;
  const SlotState* S = a.st + slot;
  if (S->status != SLOT_INIT) return;
  const LatGeom g = a.lats[S->lat];
  if (j >= g.defl_k) return;
  double acc[1] = {0.0};
  const double* vj = g.defl_V + (size_t)j * g.V;
  for (int site = threadIdx.x; site < g.V; site += NT) acc[0] += vj[site] * lap_source(g, site, S->m, S->a);
  __shared__ double sh[NT / 32];
  double t = acc[0];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int w = 0; w < NT / 32; ++w) tot += sh[w];
    a.dc[(size_t)slot * g.defl_k + j] = tot;
  }
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

// ---- per-slot scalar steps of CG (one thread, after the slot's reduction): shared by the
// lattice engine (one slot per block row) and the blocked sparse engine (all slots per block)
__device__ __forceinline__ void cg_after_init(SlotState* S, const LatGeom& g, double bb) {
  S->bnorm2 = bb;
  S->rnorm2 = bb;
  S->rmax2 = bb;
  S->rho = make_double2(bb, 0.0);
  S->iters = 0;
  S->updates = 0;
  S->need_update = 0;
  S->restart = 0;
  S->true_res2 = bb;
  S->gauss = 0.0;
  S->radau = g.quad_mu > 0.0 ? 1.0 / g.quad_mu : 0.0;
  S->status = bb > 0.0 ? SLOT_RUN : SLOT_DONE;
}

// alpha = rr / (p, A p)
__device__ __forceinline__ void cg_after_ap(SlotState* S, double pq) {
  S->alpha = make_double2(pq != 0.0 ? S->rho.x / pq : 0.0, 0.0);
  S->gauss += S->alpha.x * S->rho.x;   // Gauss rule: G_{k+1} = G_k + gamma_k ||r_k||^2
  S->restart = 0;
  S->sloppy_mv += 1;
}

// beta = rr' / rr, the Gauss-Radau coefficient, and the stopping tests
// delta2 > 0 (mixed precision): also ask for a true residual once ||r||^2 fell below delta2 times
// its largest value since the last one (reliable updates)
__device__ __forceinline__ void cg_after_xr(SlotState* S, const LatGeom& g, double rr, double tol2, int maxiter,
                                            double delta2 = 0.0) {
  const double delta = S->rho.x != 0.0 ? rr / S->rho.x : 0.0;
  S->beta = make_double2(delta, 0.0);
  S->rho = make_double2(rr, 0.0);
  S->rnorm2 = rr;
  S->rmax2 = fmax(S->rmax2, rr);
  S->iters += 1;
  if (g.quad_mu > 0.0) {   // Gauss-Radau: gt_{k+1} = (gt_k - gamma_k) / (mu (gt_k - gamma_k) + delta_{k+1})
    const double d = S->radau - S->alpha.x;
    const double den = g.quad_mu * d + delta;
    S->radau = den > 0.0 ? fmax(d, 0.0) / den : 0.0;
  }
  if (S->iters >= maxiter) {
    S->status = SLOT_FAIL;
    S->need_update = 1;
  } else if (g.quad_tol > 0.0) {   // stop on the quadrature bracket: no residual test, no restart
    if (S->radau * rr <= g.quad_tol * S->gauss || rr == 0.0 || !(rr == rr)) {
      S->true_res2 = rr;
      S->status = (rr == rr) ? SLOT_DONE : SLOT_FAIL;
    }
  } else if (rr <= tol2 * S->bnorm2 || !(rr == rr) || rr <= delta2 * S->rmax2) {
    S->need_update = 1;
  }
}

// the FP64 true residual: converged, or continue from it with p = r (keep_p: with the old p,
// the reliable update of mixed precision)
__device__ __forceinline__ void cg_after_true(SlotState* S, double rr, double tol2, bool keep_p = false) {
  S->true_res2 = rr;
  S->updates += 1;
  S->fp64_mv += 1;
  S->need_update = 0;
  if (S->status == SLOT_RUN) {
    if (rr <= tol2 * S->bnorm2) {
      S->status = SLOT_DONE;
    } else {
      S->rho = make_double2(rr, 0.0);
      S->rnorm2 = rr;
      S->rmax2 = rr;
      S->restart = keep_p ? 0 : 1;
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
    double b = lap_src(g, a, slot, site, m, pa);
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
      cg_after_init(S, g, tot[0]);
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
      cg_after_ap(S, tot[0]);
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
      cg_after_xr(S, g, tot[0], a.tol2, a.maxiter);
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
    double rv = lap_src(g, a, slot, site, m, pa) - lap_site(g, a.x + off, site);
    a.r[off + site] = rv;
    acc[0] += rv * rv;
  }
  lreduce<1, NT>(acc, part, a.gy, bx);
  if (last_block(a.cnt + slot, nparts)) {
    double tot[1];
    block_sum_partials<1, NT>(part, a.gy, nparts, tot);
    if (threadIdx.x == 0) {
      cg_after_true(S, tot[0], a.tol2);
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
    acc[0] += lap_src(g, a, slot, site, m, pa) * a.x[off + site];
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
  int big_lat = 0;   // index of the largest lattice (set by the scheduler; unused here)
  bool one_lat = false;   // one lattice in the problem (set by the scheduler; unused here)
  int defl_k = 0;
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
    defl_k = big.defl_k;
    if (defl_k) {
      HP_TRY(hp_ws(ctx, "solve.defl_c", sizeof(double) * (size_t)ns * defl_k, &p));
      a.dc = (double*)p;
    }
    return HP_OK;
  }
  hp_status init() {
    if (defl_k) {
      ProfScope ps(ctx, "k_cg_defl");
      k_cg_defl<NT><<<dim3(defl_k, nslots), NT, 0, ctx->stream>>>(a);
    }
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
  hp_status keep(const std::vector<int>&, const std::vector<SlotState>&, const SolveProblem&) {
    hp_set_error("solutions are kept for the Wilson operator only");
    return HP_EUNSUPPORTED;
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

// ------------------------------------------------------------ blocked sparse CG
// A general sparse matrix runs all B = 32 SPL slots as one block of vectors laid out
// [row][slot] (lane l of a warp owns slots l, l + 32, ...).  One warp per row reads the row's
// CSR entries once for every slot and gathers B contiguous values per entry (256 SPL bytes,
// whole sectors), where one slot per block row would re-read the matrix for every slot and
// gather single words.  Reductions: each block leaves per-slot partial sums, the last block
// to finish adds them in a fixed order and takes the scalar CG steps of every slot.
struct BArgs {
  const LatGeom* lat;
  SlotState* st;
  double *x, *r, *p, *q;   // [n][B]
  double* part;            // [B][nblk]
  unsigned int* cnt;       // one counter per reducing kernel
  int nblk;               // blocks of the matrix-vector kernels
  int nstream;            // blocks of the streaming kernels
  int pstride;            // row stride of part: max(nblk, nstream)
  double tol2;
  int maxiter;
  // mixed precision: r, p, q and the correction xl in FP32, x = xh + xl with xh in FP64
  float *xl, *rf, *pf, *qf;
  const float* val32;     // the CSR values rounded to FP32
  double delta2;          // reliable-update threshold (squared)
};

enum { BK_INIT = 0, BK_AP, BK_XR, BK_TRUE, BK_QUAD, BK_COUNT };
constexpr int BT = 256;   // threads per block of the blocked kernels

__device__ __forceinline__ bool bk_on(const SlotState* S, int kind) {
  switch (kind) {
    case BK_INIT: return S->status == SLOT_INIT;
    case BK_AP:
    case BK_XR: return S->status == SLOT_RUN;
    case BK_TRUE: return S->need_update != 0;
    default: return S->status == SLOT_DONE || S->status == SLOT_FAIL;
  }
}

template <int SPL>
__device__ __forceinline__ void bk_finish(const BArgs& a, const LatGeom& g, int kind, const double (&acc)[SPL]) {
  constexpr int B = 32 * SPL, NW = BT / 32;
  __shared__ double sh[NW][B];
  __shared__ double tot_sh[B];
  __shared__ int am_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < SPL; ++k) sh[warp][lane + 32 * k] = acc[k];
  __syncthreads();
  if (threadIdx.x < B) {
    double t = 0.0;
    for (int w = 0; w < NW; ++w) t += sh[w][threadIdx.x];
    a.part[(size_t)threadIdx.x * a.pstride + blockIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(a.cnt + kind, 1u) == (unsigned)gridDim.x - 1u;
  __syncthreads();
  if (!am_last) return;
  __threadfence();
  // warp w adds up the partials of slots w, w + NW, ...: lanes run over the blocks (coalesced
  // loads, four independent sums each), then a shuffle tree; the order is fixed
  const int nb = gridDim.x;
  for (int s = warp; s < B; s += NW) {
    const double* ps = a.part + (size_t)s * a.pstride;
    double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
    int j = lane;
    for (; j + 96 < nb; j += 128) {
      t0 += __ldcg(ps + j);
      t1 += __ldcg(ps + j + 32);
      t2 += __ldcg(ps + j + 64);
      t3 += __ldcg(ps + j + 96);
    }
    for (; j < nb; j += 32) t0 += __ldcg(ps + j);
    double t = (t0 + t1) + (t2 + t3);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) tot_sh[s] = t;
  }
  __syncthreads();
  if (threadIdx.x < B) {
    const double tot = tot_sh[threadIdx.x];
    SlotState* S = a.st + threadIdx.x;
    if (bk_on(S, kind)) {
      switch (kind) {
        case BK_INIT: cg_after_init(S, g, tot); break;
        case BK_AP: cg_after_ap(S, tot); break;
        case BK_XR: cg_after_xr(S, g, tot, a.tol2, a.maxiter, a.delta2); break;
        case BK_TRUE: cg_after_true(S, tot, a.tol2, a.xl != nullptr); break;
        default: S->q = make_double2(tot, 0.0); break;
      }
    }
  }
  if (threadIdx.x == 0) a.cnt[kind] = 0;
}

#define BK_ROWS(i) for (int i = blockIdx.x * (BT / 32) + (threadIdx.x >> 5); i < g.V; i += gridDim.x * (BT / 32))
// rows i0 + u tw, u < BR, per warp and step: a streaming kernel issues all their loads first
constexpr int BR = 4;
#define BK_ROW_BATCHES(i0, tw)                            \
  const int tw = gridDim.x * (BT / 32);                   \
  for (int i0 = blockIdx.x * (BT / 32) + (threadIdx.x >> 5); i0 < g.V; i0 += BR * tw)

// x = 0, r = p = b for the slots being filled; ||b||^2
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcg_init(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  int m[SPL], pa[SPL];
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = bk_on(S, BK_INIT);
    m[k] = S->m;
    pa[k] = S->a;
    acc[k] = 0.0;
  }
  BK_ROWS(i) {
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      if (!on[k]) continue;
      const size_t o = (size_t)i * B + lane + 32 * k;
      const double b = lap_source(g, i, m[k], pa[k]);
      a.x[o] = 0.0;
      a.r[o] = b;
      a.p[o] = b;
      acc[k] += b * b;
    }
  }
  bk_finish<SPL>(a, g, BK_INIT, acc);
}

// (A v)[i][slot] for the rows r0 .. r1-1 of one warp, handed to flush(i, value, own) row by row
// in order, with own = own_src[i][slot] (own_src may be NULL).  The rows'
// CSR entries are contiguous: the warp loads them 32 at a time (one entry per lane, coalesced;
// the next 32 are requested before the current ones are used), broadcasts each entry, and
// issues U gathers of B contiguous values before it adds them.  Each warp walks a long chain of
// dependent loads, so every load that can be issued early is.
template <int SPL, typename T, int U = 8, class Flush>
__device__ __forceinline__ void bk_spmv_rows(const LatGeom& g, const T* __restrict__ val, const T* __restrict__ v,
                                             const T* __restrict__ own_src, int r0, int r1, int lane,
                                             const bool (&on)[SPL], Flush&& flush) {
  constexpr int B = 32 * SPL;
  constexpr unsigned FULL = 0xffffffffu;
  if (r0 >= r1) return;
  int i = r0, rbase = r0;
  int rend_l = (rbase + lane < r1) ? __ldg(g.csr_rp + rbase + lane + 1) : 0x7fffffff;
  int row_end = __shfl_sync(FULL, rend_l, 0);
  T acc[SPL], own[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) acc[k] = T(0);
  auto advance = [&](int e) {   // flush every row that ends at entry e (empty rows included)
    while (i < r1 && row_end == e) {
#pragma unroll
      for (int k = 0; k < SPL; ++k) own[k] = (own_src && on[k]) ? own_src[(size_t)i * B + lane + 32 * k] : T(0);
      flush(i, acc, own);
#pragma unroll
      for (int k = 0; k < SPL; ++k) acc[k] = T(0);
      ++i;
      if (i - rbase == 32) {
        rbase = i;
        rend_l = (rbase + lane < r1) ? __ldg(g.csr_rp + rbase + lane + 1) : 0x7fffffff;
      }
      if (i < r1) row_end = __shfl_sync(FULL, rend_l, i - rbase);
    }
  };
  const int e_beg = __ldg(g.csr_rp + r0), e_fin = __ldg(g.csr_rp + r1);
  advance(e_beg);
  int c_n = e_beg + lane < e_fin ? __ldg(g.csr_ci + e_beg + lane) : 0;
  T w_n = e_beg + lane < e_fin ? __ldg(val + e_beg + lane) : T(0);
  for (int e0 = e_beg; e0 < e_fin; e0 += 32) {
    const int nb = min(32, e_fin - e0);
    const int c_l = c_n;
    const T w_l = w_n;
    const int en = e0 + 32 + lane;   // the next 32 entries, requested now
    c_n = en < e_fin ? __ldg(g.csr_ci + en) : 0;
    w_n = en < e_fin ? __ldg(val + en) : T(0);
    for (int j0 = 0; j0 < nb; j0 += U) {
      T gv[U][SPL];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int c = __shfl_sync(FULL, c_l, j0 + u);   // lanes past nb hold row 0: in bounds, unused
        const T* vj = v + (size_t)c * B + lane;
#pragma unroll
        for (int k = 0; k < SPL; ++k) gv[u][k] = (on[k] && j0 + u < nb) ? vj[32 * k] : T(0);
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        if (j0 + u < nb) {
          const T w = __shfl_sync(FULL, w_l, j0 + u);
#pragma unroll
          for (int k = 0; k < SPL; ++k) acc[k] += w * gv[u][k];
          advance(e0 + j0 + u + 1);
        }
      }
    }
  }
}

// the contiguous rows of warp number gw of tw warps
__device__ __forceinline__ void bk_warp_rows(int n, int& r0, int& r1) {
  const int tw = gridDim.x * (BT / 32), gw = blockIdx.x * (BT / 32) + (threadIdx.x >> 5);
  const int chunk = (n + tw - 1) / tw;
  r0 = min(n, gw * chunk);
  r1 = min(n, r0 + chunk);
}

// q = A p ; (p, q)
template <int SPL>
__global__ void __launch_bounds__(BT, SPL == 1 ? 4 : (SPL == 2 ? 3 : 2)) k_bcg_ap(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    on[k] = bk_on(a.st + lane + 32 * k, BK_AP);
    acc[k] = 0.0;
  }
  int r0, r1;
  bk_warp_rows(g.V, r0, r1);
  bk_spmv_rows<SPL, double>(g, g.csr_val, a.p, a.p, r0, r1, lane, on, [&](int i, const double (&qv)[SPL], const double (&pv)[SPL]) {
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      if (!on[k]) continue;
      a.q[(size_t)i * B + lane + 32 * k] = qv[k];
      acc[k] += pv[k] * qv[k];
    }
  });
  bk_finish<SPL>(a, g, BK_AP, acc);
}

// x += alpha p ; r -= alpha q ; (r, r)
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcg_xr(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  double al[SPL], acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = bk_on(S, BK_XR);
    al[k] = S->alpha.x;
    acc[k] = 0.0;
  }
  double* __restrict__ x = a.x;
  double* __restrict__ r = a.r;
  const double* __restrict__ p = a.p;
  const double* __restrict__ q = a.q;
  BK_ROW_BATCHES(i0, tw) {   // loads of BR rows first, then the updates: BR x 4 SPL loads in flight
    double xv[BR][SPL], pv[BR][SPL], qv[BR][SPL], rv[BR][SPL];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        xv[u][k] = x[o];
        pv[u][k] = p[o];
        qv[u][k] = q[o];
        rv[u][k] = r[o];
      }
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        x[o] = xv[u][k] + al[k] * pv[u][k];
        const double rn = rv[u][k] - al[k] * qv[u][k];
        r[o] = rn;
        acc[k] += rn * rn;
      }
  }
  bk_finish<SPL>(a, g, BK_XR, acc);
}

// p = r + beta p
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcg_p(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  double be[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = S->status == SLOT_RUN;
    be[k] = S->restart ? 0.0 : S->beta.x;
  }
  double* __restrict__ p = a.p;
  const double* __restrict__ r = a.r;
  BK_ROW_BATCHES(i0, tw) {
    double pv[BR][SPL], rv[BR][SPL];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        pv[u][k] = p[o];
        rv[u][k] = r[o];
      }
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        p[(size_t)i * B + lane + 32 * k] = rv[u][k] + be[k] * pv[u][k];
      }
  }
}

// q = b . x for the finished slots
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcg_quad(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  int m[SPL], pa[SPL];
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = bk_on(S, BK_QUAD);
    m[k] = S->m;
    pa[k] = S->a;
    acc[k] = 0.0;
  }
  BK_ROWS(i) {
#pragma unroll
    for (int k = 0; k < SPL; ++k)
      if (on[k]) acc[k] += lap_source(g, i, m[k], pa[k]) * a.x[(size_t)i * B + lane + 32 * k];
  }
  bk_finish<SPL>(a, g, BK_QUAD, acc);
}

// ---- mixed precision (FP32 iteration, FP64 reliable updates): the matrix-vector product,
// the recurrences and the per-lane dot products in FP32; ||b||^2, the block sums and the true
// residual b - A (xh + xl) in FP64.  A reliable update folds xl into xh, recomputes r in FP64
// and keeps p.

// xh = 0, xl = 0, r = p = b
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcm_init(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  int m[SPL], pa[SPL];
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = bk_on(S, BK_INIT);
    m[k] = S->m;
    pa[k] = S->a;
    acc[k] = 0.0;
  }
  BK_ROWS(i) {
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      if (!on[k]) continue;
      const size_t o = (size_t)i * B + lane + 32 * k;
      const double b = lap_source(g, i, m[k], pa[k]);
      a.x[o] = 0.0;
      a.xl[o] = 0.0f;
      a.rf[o] = (float)b;
      a.pf[o] = (float)b;
      acc[k] += b * b;
    }
  }
  bk_finish<SPL>(a, g, BK_INIT, acc);
}

// q = A p, (p, q) in FP32
template <int SPL>
__global__ void __launch_bounds__(BT, SPL <= 2 ? 4 : 2) k_bcm_ap(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  float accf[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    on[k] = bk_on(a.st + lane + 32 * k, BK_AP);
    accf[k] = 0.0f;
  }
  int r0, r1;
  bk_warp_rows(g.V, r0, r1);
  bk_spmv_rows<SPL, float, 16>(g, a.val32, a.pf, a.pf, r0, r1, lane, on,
                           [&](int i, const float (&qv)[SPL], const float (&pv)[SPL]) {
#pragma unroll
                             for (int k = 0; k < SPL; ++k) {
                               if (!on[k]) continue;
                               a.qf[(size_t)i * B + lane + 32 * k] = qv[k];
                               accf[k] = fmaf(pv[k], qv[k], accf[k]);
                             }
                           });
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) acc[k] = accf[k];
  bk_finish<SPL>(a, g, BK_AP, acc);
}

// xl += alpha p, r -= alpha q, (r, r) in FP32
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcm_xr(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  float al[SPL], accf[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = bk_on(S, BK_XR);
    al[k] = (float)S->alpha.x;
    accf[k] = 0.0f;
  }
  float* __restrict__ xl = a.xl;
  float* __restrict__ rf = a.rf;
  const float* __restrict__ pf = a.pf;
  const float* __restrict__ qf = a.qf;
  BK_ROW_BATCHES(i0, tw) {
    float xv[BR][SPL], pv[BR][SPL], qv[BR][SPL], rv[BR][SPL];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        xv[u][k] = xl[o];
        pv[u][k] = pf[o];
        qv[u][k] = qf[o];
        rv[u][k] = rf[o];
      }
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        xl[o] = fmaf(al[k], pv[u][k], xv[u][k]);
        const float rn = fmaf(-al[k], qv[u][k], rv[u][k]);
        rf[o] = rn;
        accf[k] = fmaf(rn, rn, accf[k]);
      }
  }
  double acc[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) acc[k] = accf[k];
  bk_finish<SPL>(a, g, BK_XR, acc);
}

// reliable update, first half: xh += xl, xl = 0 for the slots that asked for a true residual
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcm_fold(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  bool any = false;
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    on[k] = bk_on(a.st + lane + 32 * k, BK_TRUE);
    any |= on[k];
  }
  if (!__syncthreads_or(any)) return;
  BK_ROWS(i) {
#pragma unroll
    for (int k = 0; k < SPL; ++k) {
      if (!on[k]) continue;
      const size_t o = (size_t)i * B + lane + 32 * k;
      a.x[o] += (double)a.xl[o];
      a.xl[o] = 0.0f;
    }
  }
}

// p = r + beta p in FP32
template <int SPL>
__global__ void __launch_bounds__(BT) k_bcm_p(BArgs a) {
  constexpr int B = 32 * SPL;
  const LatGeom g = *a.lat;
  const int lane = threadIdx.x & 31;
  bool on[SPL];
  float be[SPL];
#pragma unroll
  for (int k = 0; k < SPL; ++k) {
    const SlotState* S = a.st + lane + 32 * k;
    on[k] = S->status == SLOT_RUN;
    be[k] = S->restart ? 0.0f : (float)S->beta.x;
  }
  float* __restrict__ pf = a.pf;
  const float* __restrict__ rf = a.rf;
  BK_ROW_BATCHES(i0, tw) {
    float pv[BR][SPL], rv[BR][SPL];
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        const size_t o = (size_t)i * B + lane + 32 * k;
        pv[u][k] = pf[o];
        rv[u][k] = rf[o];
      }
#pragma unroll
    for (int u = 0; u < BR; ++u)
#pragma unroll
      for (int k = 0; k < SPL; ++k) {
        const int i = i0 + u * tw;
        if (i >= g.V || !on[k]) continue;
        pf[(size_t)i * B + lane + 32 * k] = fmaf(be[k], pv[u][k], rv[u][k]);
      }
  }
}

// True residual r = b - A x in FP64 for the slots that asked for one, one thread per row and a
// grid row per slot (most iterations one slot or none asks: a warp per row over all slots would
// walk the whole matrix for a single lane).  MIXED: r is stored in FP32 for the iteration and
// the old p is kept.
template <int SPL, bool MIXED>
__global__ void __launch_bounds__(256) k_btrue_slot(BArgs a, double* __restrict__ part, unsigned int* __restrict__ cnt) {
  constexpr int B = 32 * SPL;
  const int slot = blockIdx.y;
  SlotState* S = a.st + slot;
  if (!S->need_update) return;
  const LatGeom g = *a.lat;
  const int m = S->m, pa = S->a;
  double acc[1] = {0.0};
  for (int i = blockIdx.x * 256 + threadIdx.x; i < g.V; i += gridDim.x * 256) {
    double ax = 0.0;
    const int e1 = __ldg(g.csr_rp + i + 1);
    for (int e = __ldg(g.csr_rp + i); e < e1; ++e)
      ax += __ldg(g.csr_val + e) * a.x[(size_t)__ldg(g.csr_ci + e) * B + slot];
    const double rv = lap_source(g, i, m, pa) - ax;
    if (MIXED)
      a.rf[(size_t)i * B + slot] = (float)rv;
    else
      a.r[(size_t)i * B + slot] = rv;
    acc[0] += rv * rv;
  }
  lreduce<1, 256>(acc, part + (size_t)slot * gridDim.x, 0, blockIdx.x);
  if (last_block(cnt + slot, gridDim.x)) {
    double tot[1];
    block_sum_partials<1, 256>(part + (size_t)slot * gridDim.x, 0, gridDim.x, tot);
    if (threadIdx.x == 0) {
      cg_after_true(S, tot[0], a.tol2, MIXED);
      cnt[slot] = 0;
    }
  }
}

__global__ void k_to_f32(const double* __restrict__ in, long long n, float* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)in[i];
}

template <int SPL, bool MIXED>
struct BlockedSparseEngine {
  static constexpr int B = 32 * SPL;
  static constexpr int GROUP_MAX = B;   // the schedule's slot count is exactly B
  int kernels_per_iteration() const { return MIXED ? 5 : 4; }
  hp_ctx* ctx;
  BArgs a;
  int big_lat = 0;          // index of the largest lattice (set by the scheduler; unused here)
  bool one_lat = false;     // one lattice in the problem (set by the scheduler; unused here)
  int ntrue = 1;            // row blocks of the true-residual kernel (per slot)
  double* tpart = nullptr;  // its partial sums [B][ntrue]
  unsigned int* tcnt = nullptr;
  long long nnz = 0;
  double delta = 0.0;
  int group() const { return 1; }
  hp_status setup(int ns, int Vmax, const LatGeom* lats_dev, SlotState* st, const hp_solver_opts& o, double tol,
                  double, const LatGeom&) {
    if (ns != B) {
      hp_set_error("blocked sparse CG: %d slots for a block of %d", ns, B);
      return HP_EINVAL;
    }
    memset(&a, 0, sizeof(a));
    a.lat = lats_dev;
    a.st = st;
    // one resident wave of the matrix-vector kernel (a second, partial wave would idle most SMs)
    int occ = 0;
    HP_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, MIXED ? (const void*)k_bcm_ap<SPL>
                                                                       : (const void*)k_bcg_ap<SPL>, BT, 0));
    const long long rows_blocks = ((long long)Vmax + BT / 32 - 1) / (BT / 32);   // one row per warp at least
    auto wave = [&](int blocks_per_sm) {
      return (int)std::max(1LL, std::min<long long>(rows_blocks, (long long)ctx->num_sms * std::max(blocks_per_sm, 1)));
    };
    a.nblk = wave(occ);
    a.nstream = wave(2048 / BT);
    a.pstride = std::max(a.nblk, a.nstream);
    void* p = nullptr;
    ntrue = (int)std::max(1LL, std::min<long long>(((long long)Vmax + 255) / 256, (long long)ctx->num_sms * 2));
    HP_TRY(hp_ws(ctx, "bcg.tpart", sizeof(double) * (size_t)B * ntrue, &p));
    tpart = (double*)p;
    HP_TRY(hp_ws(ctx, "bcg.tcnt", sizeof(unsigned int) * B, &p));
    tcnt = (unsigned int*)p;
    HP_CUDA(cudaMemsetAsync(tcnt, 0, sizeof(unsigned int) * B, ctx->stream));
    HP_TRY(hp_ws(ctx, "bcg.part", sizeof(double) * (size_t)B * a.pstride, &p));
    a.part = (double*)p;
    HP_TRY(hp_ws(ctx, "bcg.cnt", sizeof(unsigned int) * BK_COUNT, &p));
    a.cnt = (unsigned int*)p;
    HP_CUDA(cudaMemsetAsync(a.cnt, 0, sizeof(unsigned int) * BK_COUNT, ctx->stream));
    const size_t fb = sizeof(double) * (size_t)B * Vmax;
    double** v[4] = {&a.x, &a.r, &a.p, &a.q};
    const char* names[4] = {"solve.lx", "solve.lr", "solve.lp", "solve.lq"};
    for (int k = 0; k < (MIXED ? 1 : 4); ++k) {
      HP_TRY(hp_ws(ctx, names[k], fb, &p));
      *v[k] = (double*)p;
      HP_CUDA(cudaMemsetAsync(p, 0, fb, ctx->stream));   // columns of idle slots stay finite
    }
    if (MIXED) {
      const size_t fs = sizeof(float) * (size_t)B * Vmax;
      float** vf[4] = {&a.xl, &a.rf, &a.pf, &a.qf};
      const char* nf[4] = {"solve.xl32", "solve.r32", "solve.p32", "solve.q32"};
      for (int k = 0; k < 4; ++k) {
        HP_TRY(hp_ws(ctx, nf[k], fs, &p));
        *vf[k] = (float*)p;
        HP_CUDA(cudaMemsetAsync(p, 0, fs, ctx->stream));
      }
      LatGeom g;   // the CSR values in FP32
      HP_CUDA(cudaMemcpyAsync(&g, lats_dev, sizeof(LatGeom), cudaMemcpyDeviceToHost, ctx->stream));
      HP_CUDA(cudaStreamSynchronize(ctx->stream));
      int e_end = 0;
      HP_CUDA(cudaMemcpyAsync(&e_end, g.csr_rp + g.V, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
      HP_CUDA(cudaStreamSynchronize(ctx->stream));
      nnz = e_end;
      HP_TRY(hp_ws(ctx, "bcg.val32", sizeof(float) * (size_t)std::max(nnz, 1LL), &p));
      a.val32 = (const float*)p;
      if (nnz) {
        ProfScope ps(ctx, "k_to_f32");
        k_to_f32<<<blocks_for(ctx, nnz, 256), 256, 0, ctx->stream>>>(g.csr_val, nnz, (float*)p);
      }
      HP_LAUNCH_CHECK();
      // default threshold: a true residual after every 10^5 reduction (measured on the renumbered
      // 64^3 grid: 1e-3 -> 4.0 updates per solve, 1e-4 -> 3.0, 1e-5 -> 2.1 with the FP64 iteration
      // count, 1e-6 -> 2.0 but 1.7% more iterations)
      const double d = o.delta > 0.0 ? o.delta : 1e-5;
      a.delta2 = d * d;
    }
    a.tol2 = tol * tol;
    a.maxiter = o.maxiter > 0 ? o.maxiter : 10000;
    return HP_OK;
  }
  hp_status init() {
    if (MIXED) {
      ProfScope ps(ctx, "k_bcm_init");
      k_bcm_init<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a);
    } else {
      ProfScope ps(ctx, "k_bcg_init");
      k_bcg_init<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status iteration() {
    if (MIXED) {
      { ProfScope ps(ctx, "k_bcm_ap"); k_bcm_ap<SPL><<<a.nblk, BT, 0, ctx->stream>>>(a); }
      { ProfScope ps(ctx, "k_bcm_xr"); k_bcm_xr<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
      { ProfScope ps(ctx, "k_bcm_fold"); k_bcm_fold<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
      {
        ProfScope ps(ctx, "k_btrue_slot");
        k_btrue_slot<SPL, true><<<dim3(ntrue, B), 256, 0, ctx->stream>>>(a, tpart, tcnt);
      }
      { ProfScope ps(ctx, "k_bcm_p"); k_bcm_p<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
      HP_LAUNCH_CHECK();
      return HP_OK;
    }
    { ProfScope ps(ctx, "k_bcg_ap"); k_bcg_ap<SPL><<<a.nblk, BT, 0, ctx->stream>>>(a); }
    { ProfScope ps(ctx, "k_bcg_xr"); k_bcg_xr<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
    {
      ProfScope ps(ctx, "k_btrue_slot");
      k_btrue_slot<SPL, false><<<dim3(ntrue, B), 256, 0, ctx->stream>>>(a, tpart, tcnt);
    }
    { ProfScope ps(ctx, "k_bcg_p"); k_bcg_p<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status keep(const std::vector<int>&, const std::vector<SlotState>&, const SolveProblem&) {
    hp_set_error("solutions are kept for the Wilson operator only");
    return HP_EUNSUPPORTED;
  }
  hp_status harvest(const std::vector<int>&, const SolveProblem&, int*) {
    { ProfScope ps(ctx, "k_bcg_quad"); k_bcg_quad<SPL><<<a.nstream, BT, 0, ctx->stream>>>(a); }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
};

#include "hp_schedule.cuh"

template <int SPL, bool MIXED>
static hp_status run_blocked(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  BlockedSparseEngine<SPL, MIXED> e{ctx};
  return run_schedule(ctx, e, pb, res, 12, 0.0);
}

hp_status hp_solve_laplace(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  if (pb.lats.size() == 1 && pb.lats[0].csr_rp && !pb.want_grad) {
    // blocked engine: B slots (rhs_block rounded up to 32, 64 or 128; automatic: 64, the fastest
    // on the renumbered 64^3 grid matrix in both precisions)
    const int want = pb.opts.rhs_block > 0 ? pb.opts.rhs_block : 64;
    const bool mixed = pb.opts.precision == HP_PREC_MIXED_FP32;
    pb.opts.rhs_block = want <= 32 ? 32 : (want <= 64 ? 64 : 128);
    if (mixed) {
      if (want <= 32) return run_blocked<1, true>(ctx, pb, res);
      if (want <= 64) return run_blocked<2, true>(ctx, pb, res);
      return run_blocked<4, true>(ctx, pb, res);
    }
    if (want <= 32) return run_blocked<1, false>(ctx, pb, res);
    if (want <= 64) return run_blocked<2, false>(ctx, pb, res);
    return run_blocked<4, false>(ctx, pb, res);
  }
  LaplaceEngine e{ctx};
  return run_schedule(ctx, e, pb, res, 12, 0.0);
}
