// Deflated hierarchical probing of the Wilson matrix (the variance reduction the paper's
// conclusions pair with probing), by a correction of the plain quadratures.
//
// With singular triplets D v_j = sigma_j u_j (right vectors v_j, left vectors u_j, each set
// orthonormal; D^-1 u_j = v_j / sigma_j),
//   Tr D^-1 = sum_j (u_j^H v_j) / sigma_j + Tr(D^-1 (I - U U^H)),
// and the probed part of vector m, sum_a v_{m,a}^H D^-1 (I - U U^H) v_{m,a}, equals the plain
// quadrature q_m minus
//   c_m = sum_a sum_j (v_{m,a}^H v_j) (u_j^H v_{m,a}) / sigma_j.
// Eigenpairs Q w_j = lambda_j w_j of the Hermitian Q = gamma_5 D are such triplets:
// v_j = w_j, u_j = sign(lambda_j) gamma_5 w_j, sigma_j = |lambda_j|.  The solves are the plain
// ones; the correction needs the projections of the first s vectors onto the v_j and u_j only.
// The first 2^kb hierarchical vectors are constant on the 2^kb blocks of consecutive hierarchical
// positions (the top kb binary digits), so with the block sums
//   B_{j,a}(b) = sum over the sites x of block b of z_0(x) w(x, a)     (w = v_j or u_j)
// the projections are 2^kb-point Walsh-Hadamard sums, v_{m,a}^H w = sum_b (-1)^{|b & rev(m)|} B(b);
// past the binary levels every hierarchical position is its own block and the phases are the
// full mixed-radix ones.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr int WT = 256;

__global__ void k_wd_iperm(const uint32_t* __restrict__ loc, int V, int* __restrict__ iperm) {
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < V; x += gridDim.x * blockDim.x) iperm[loc[x]] = x;
}

__device__ __forceinline__ double wd_z0(unsigned long long seed, int x) {
  return (seed && (splitmix64_at(seed, (unsigned long long)x) >> 63)) ? -1.0 : 1.0;
}

// the hierarchical phase (integer, period P) of vector m at hierarchical position loc, without z_0:
// the binary levels by bit reversal, then the three-colour and final Fourier levels
__device__ __forceinline__ int wd_phase(const LatGeom& g, uint32_t loc, uint32_t m) {
  uint32_t lb = loc, w = 0;
  if (g.Q > 1) {
    lb = loc / (uint32_t)g.Q;
    w = loc - lb * (uint32_t)g.Q;
  }
  int ph = 0;
  uint32_t hi = m;
  if (g.K > 0) {
    const uint32_t ebin = m & ((1u << g.K) - 1u);
    hi = m >> g.K;
    const uint32_t col = __brev(ebin) >> (32 - g.K);
    ph = (__popc(lb & col) & 1) * (g.P >> 1);
  }
  if (hi > 0 && g.R > 0) {
    const uint32_t e3 = hi % 3u, ef = hi / 3u;
    const uint32_t C = w / (uint32_t)g.R, r = w - C * (uint32_t)g.R;
    ph += (g.P / 3) * (int)((C * e3) % 3u);
    ph += (g.P / g.R) * (int)((unsigned long long)r * ef % (unsigned long long)g.R);
  }
  return ph % g.P;
}

// sum of NV doubles over the block in a fixed order (warp shuffles, then warps in order); the
// result lands in thread 0
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[WT / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NV; ++i)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[i] += __shfl_down_sync(0xffffffffu, v[i], o);
  if (lane == 0)
#pragma unroll
    for (int i = 0; i < NV; ++i) sh[warp][i] = v[i];
  __syncthreads();
  if (threadIdx.x == 0)
    for (int i = 0; i < NV; ++i) {
      double t = 0.0;
      for (int u = 0; u < (int)(blockDim.x >> 5); ++u) t += sh[u][i];
      v[i] = t;
    }
}

// B[(j * 12 + a) * nblk + blk] = sum over positions blk * bs .. (blk + 1) * bs - 1 of z0(x) w_j(x, a)
__global__ void __launch_bounds__(WT) k_wd_blocksum(const double2* __restrict__ W, const int* __restrict__ iperm,
                                                    int V, long long bs, int nblk, unsigned long long seed,
                                                    double2* __restrict__ B) {
  const int blk = blockIdx.x, j = blockIdx.y;
  double acc[24];
#pragma unroll
  for (int i = 0; i < 24; ++i) acc[i] = 0.0;
  for (long long t = threadIdx.x; t < bs; t += blockDim.x) {
    const int x = iperm[(long long)blk * bs + t];
    const double z = wd_z0(seed, x);
    const double2* w = W + ((size_t)j * V + x) * 12;
#pragma unroll
    for (int a = 0; a < 12; ++a) {
      const double2 e = w[a];
      acc[2 * a] = fma(z, e.x, acc[2 * a]);
      acc[2 * a + 1] = fma(z, e.y, acc[2 * a + 1]);
    }
  }
  block_sum<24>(acc);
  if (threadIdx.x == 0)
    for (int a = 0; a < 12; ++a) B[((size_t)j * 12 + a) * nblk + blk] = make_double2(acc[2 * a], acc[2 * a + 1]);
}

// q[m] -= sum_{j, a} (v_{m,a}^H v_j) conj(v_{m,a}^H u_j) / sigma_j, one block per vector m, from the block
// sums of the right (BR) and left (BL) vectors; kb >= 0: the 2^kb binary blocks, kb < 0: every
// position its own block (full phases)
__global__ void __launch_bounds__(WT) k_wd_coef(const double2* __restrict__ BR, const double2* __restrict__ BL,
                                                int nblk, int k, const double* __restrict__ sigma, LatGeom g, int kb,
                                                double2* __restrict__ q) {
  const int m = blockIdx.x;
  double part[2] = {0.0, 0.0};
  const uint32_t rm = kb > 0 ? (__brev((uint32_t)m) >> (32 - kb)) : 0u;
  for (int ja = threadIdx.x; ja < 12 * k; ja += blockDim.x) {
    const double2* br = BR + (size_t)ja * nblk;
    const double2* bl = BL + (size_t)ja * nblk;
    double rr = 0.0, ri = 0.0, lr = 0.0, li = 0.0;
    if (kb >= 0) {
      for (int b = 0; b < nblk; ++b) {
        const double sg = (__popc((uint32_t)b & rm) & 1) ? -1.0 : 1.0;
        rr = fma(sg, br[b].x, rr);
        ri = fma(sg, br[b].y, ri);
        lr = fma(sg, bl[b].x, lr);
        li = fma(sg, bl[b].y, li);
      }
    } else {
      for (int b = 0; b < nblk; ++b) {   // conj(z_m) B: (cos - i sin)(B.x + i B.y)
        const double2 z = g.ptab[wd_phase(g, (uint32_t)b, (uint32_t)m)];
        rr += z.x * br[b].x + z.y * br[b].y;
        ri += z.x * br[b].y - z.y * br[b].x;
        lr += z.x * bl[b].x + z.y * bl[b].y;
        li += z.x * bl[b].y - z.y * bl[b].x;
      }
    }
    const double s = 1.0 / sigma[ja / 12];
    part[0] += s * (rr * lr + ri * li);   // (v^H v_j) conj(v^H u_j)
    part[1] += s * (ri * lr - rr * li);
  }
  block_sum<2>(part);
  if (threadIdx.x == 0) {
    q[m].x -= part[0];
    q[m].y -= part[1];
  }
}

// e[j] = u_j^H v_j, one block per j; then out = sum_j e_j / sigma_j (complex) in one thread, in order
__global__ void __launch_bounds__(WT) k_wd_uv(const double2* __restrict__ R, const double2* __restrict__ L, int V,
                                              double2* __restrict__ e) {
  const int j = blockIdx.x;
  double acc[2] = {0.0, 0.0};
  const double2* r = R + (size_t)j * V * 12;
  const double2* l = L + (size_t)j * V * 12;
  for (long long t = threadIdx.x; t < 12LL * V; t += blockDim.x) {
    acc[0] += l[t].x * r[t].x + l[t].y * r[t].y;
    acc[1] += l[t].x * r[t].y - l[t].y * r[t].x;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) e[j] = make_double2(acc[0], acc[1]);
}

__global__ void k_wd_exact(const double2* __restrict__ e, const double* __restrict__ sigma, int k,
                           double* __restrict__ out) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < k; ++j) {
    re += e[j].x / sigma[j];
    im += e[j].y / sigma[j];
  }
  out[0] = re;
  out[1] = im;
}

// the triplets of gamma_5 eigenpairs: L[j] = sign(lambda_j) gamma_5 W[j], sigma_j = |lambda_j|
__global__ void k_wd_gamma5_left(const double2* __restrict__ W, const double* __restrict__ lam, int V, int k,
                                 double2* __restrict__ L, double* __restrict__ sigma) {
  const long long total = 12LL * V * k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(t / (12LL * V));
    const double s = (lam[j] < 0.0 ? -1.0 : 1.0) * ((t % 12) >= 6 ? -1.0 : 1.0);
    L[t] = make_double2(s * W[t].x, s * W[t].y);
    if (t % (12LL * V) == 0) sigma[j] = fabs(lam[j]);
  }
}

}  // namespace

// q (device, complex [s_max], the plain quadratures) -> the deflated ones; exact_dev[0, 1] = sum_j
// (u_j^H v_j) / sigma_j.  R, L: device, complex [k][V][4][3] (right and left vectors); sigma: device [k].
hp_status hp_wilson_deflation(hp_ctx* ctx, const LatGeom& g, int k, const double2* R, const double2* L,
                              const double* sigma, int64_t s_max, double2* q, double* exact_dev) {
  if (g.paths || g.probe_kind != HP_PROBE_HIERARCHICAL || !g.loc) {
    hp_set_error("deflated Wilson probing uses the hierarchical vectors of a lattice");
    return HP_EUNSUPPORTED;
  }
  const int V = g.V;
  int kb = -1;
  long long nblk = V, bs = 1;
  if (s_max <= (1LL << g.K)) {   // the binary levels resolve the vectors: 2^kb blocks of positions
    kb = 0;
    while ((1LL << kb) < s_max) ++kb;
    nblk = 1LL << kb;
    bs = (long long)V / nblk;
  }
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "wdefl.iperm", sizeof(int) * (size_t)V, &p));
  int* iperm = (int*)p;
  HP_TRY(hp_ws(ctx, "wdefl.BR", sizeof(double2) * (size_t)k * 12 * nblk, &p));
  double2* BR = (double2*)p;
  HP_TRY(hp_ws(ctx, "wdefl.BL", sizeof(double2) * (size_t)k * 12 * nblk, &p));
  double2* BL = (double2*)p;
  HP_TRY(hp_ws(ctx, "wdefl.e", sizeof(double2) * (size_t)k, &p));
  double2* e = (double2*)p;
  const dim3 gb((unsigned)nblk, (unsigned)k);
  const int tb = bs >= WT ? WT : 32;
  {
    ProfScope ps(ctx, "k_wd_blocksum");
    k_wd_iperm<<<blocks_for(ctx, V, 256), 256, 0, ctx->stream>>>(g.loc, V, iperm);
    k_wd_blocksum<<<gb, tb, 0, ctx->stream>>>(R, iperm, V, bs, (int)nblk, g.z0_seed, BR);
    k_wd_blocksum<<<gb, tb, 0, ctx->stream>>>(L, iperm, V, bs, (int)nblk, g.z0_seed, BL);
  }
  HP_LAUNCH_CHECK();
  {
    ProfScope ps(ctx, "k_wd_coef");
    k_wd_coef<<<(unsigned)s_max, WT, 0, ctx->stream>>>(BR, BL, (int)nblk, k, sigma, g, kb, q);
  }
  HP_LAUNCH_CHECK();
  k_wd_uv<<<k, WT, 0, ctx->stream>>>(R, L, V, e);
  k_wd_exact<<<1, 1, 0, ctx->stream>>>(e, sigma, k, exact_dev);
  HP_LAUNCH_CHECK();
  return HP_OK;
}

// the same with gamma_5 eigenpairs (W, lambda): their triplets formed on the device
hp_status hp_wilson_deflation_gamma5(hp_ctx* ctx, const LatGeom& g, int k, const double2* W, const double* lam,
                                     int64_t s_max, double2* q, double* exact_dev) {
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "wdefl.L", sizeof(double2) * 12 * (size_t)k * g.V, &p));
  double2* L = (double2*)p;
  HP_TRY(hp_ws(ctx, "wdefl.sigma", sizeof(double) * (size_t)k, &p));
  double* sigma = (double*)p;
  k_wd_gamma5_left<<<blocks_for(ctx, 12LL * g.V * k, 256), 256, 0, ctx->stream>>>(W, lam, g.V, k, L, sigma);
  HP_LAUNCH_CHECK();
  return hp_wilson_deflation(ctx, g, k, W, L, sigma, s_max, q, exact_dev);
}
