// The lowest eigenpairs of the shifted Laplacian (the modes that deflated probing removes exactly;
// the paper's conclusions name deflation as the step after probing) by Chebyshev-filtered subspace
// iteration on a block of b = k + guard vectors:
//   1. X <- p(A) X, p the Chebyshev polynomial of degree m on the damped interval [theta_b, l_max]
//      (theta_b the largest Ritz value of the block, l_max an upper bound of the spectrum), scaled
//      so that the end of the wanted interval keeps its size (three-term recurrence);
//   2. orthonormalise X (shifted Cholesky QR once, then Cholesky QR twice);
//   3. Rayleigh-Ritz: H = X^T A X (b x b), H = W diag(theta) W^T on the host (cyclic Jacobi),
//      X <- X W;
//   4. stop when the k lowest pairs have ||A x - theta x|| <= tol theta.
// Everything on the device is FP64: the Laplacian stencil (hp_apply_laplace), the recurrence, the
// Gram matrices (32 x 32 tiles of X^T Y over site chunks, partial sums added in a fixed order) and
// the block rotations X W; the host works on b x b matrices only.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "hp_internal.h"

hp_status hp_apply_laplace(hp_ctx* ctx, LatGeom g, int nrhs, const double* in, double* out);

namespace {

constexpr int GT = 32;          // Gram tile (GT x GT entries per block)
constexpr int GCH = 32;         // sites per shared-memory chunk
constexpr int CJ = 16;          // outputs per thread of the block rotation

// X[j][s] = uniform in [-1, 1) from output number j V + s of SplitMix64 seeded with `seed`
__global__ void k_eig_fill(double* __restrict__ X, long long n, unsigned long long seed) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x)
    X[t] = (double)(splitmix64_at(seed, (unsigned long long)t) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

// out = a P + c Q + e R, elementwise (R may be null when e = 0)
__global__ void k_eig_lincomb(double* __restrict__ out, const double* __restrict__ P, const double* __restrict__ Q,
                              const double* __restrict__ R, double a, double c, double e, long long n) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
    double v = a * P[t] + c * Q[t];
    if (R) v += e * R[t];
    out[t] = v;
  }
}

// partial Gram matrices: part[bx][i][j] = sum over the sites of block column bx of X[i][s] Y[j][s]
// for the GT x GT tile (blockIdx.y) of (i, j); 16 x 16 threads, 2 x 2 entries each
__global__ void __launch_bounds__(256) k_eig_gram(const double* __restrict__ X, const double* __restrict__ Y,
                                                  int V, int b, int sites_per_block, double* __restrict__ part) {
  __shared__ double xs[GT][GCH + 1], ys[GT][GCH + 1];
  const int ntj = (b + GT - 1) / GT;
  const int i0 = (blockIdx.y / ntj) * GT, j0 = (blockIdx.y % ntj) * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  const long long s_begin = (long long)blockIdx.x * sites_per_block;
  const long long s_end = std::min<long long>(V, s_begin + sites_per_block);
  for (long long s0 = s_begin; s0 < s_end; s0 += GCH) {
    for (int e = threadIdx.x; e < GT * GCH; e += 256) {
      const int r = e / GCH, c = e % GCH;
      const long long s = s0 + c;
      xs[r][c] = (i0 + r < b && s < s_end) ? X[(size_t)(i0 + r) * V + s] : 0.0;
      ys[r][c] = (j0 + r < b && s < s_end) ? Y[(size_t)(j0 + r) * V + s] : 0.0;
    }
    __syncthreads();
#pragma unroll 8
    for (int c = 0; c < GCH; ++c) {
      const double x0 = xs[2 * ty][c], x1 = xs[2 * ty + 1][c];
      const double y0 = ys[2 * tx][c], y1 = ys[2 * tx + 1][c];
      acc[0][0] = fma(x0, y0, acc[0][0]);
      acc[0][1] = fma(x0, y1, acc[0][1]);
      acc[1][0] = fma(x1, y0, acc[1][0]);
      acc[1][1] = fma(x1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  double* p = part + (size_t)blockIdx.x * b * b;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + 2 * ty + u, j = j0 + 2 * tx + v;
      if (i < b && j < b) p[(size_t)i * b + j] = acc[u][v];
    }
}

// G[e] = sum_bx part[bx][e], in block order (deterministic)
__global__ void k_eig_gram_sum(const double* __restrict__ part, int nbx, int bb, double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < bb; e += gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < nbx; ++k) t += part[(size_t)k * bb + e];
    G[e] = t;
  }
}

// Z[j][s] = sum_i X[i][s] W[i][j] for the CJ outputs j of blockIdx.y (W row-major b x b)
__global__ void k_eig_rotate(const double* __restrict__ X, const double* __restrict__ W, int V, int b,
                             double* __restrict__ Z) {
  const int j0 = blockIdx.y * CJ;
  for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < V; s += (long long)gridDim.x * blockDim.x) {
    double acc[CJ];
#pragma unroll
    for (int j = 0; j < CJ; ++j) acc[j] = 0.0;
    for (int i = 0; i < b; ++i) {
      const double x = X[(size_t)i * V + s];
      const double* w = W + (size_t)i * b + j0;
#pragma unroll
      for (int j = 0; j < CJ; ++j)
        if (j0 + j < b) acc[j] = fma(x, __ldg(w + j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < CJ; ++j)
      if (j0 + j < b) Z[(size_t)(j0 + j) * V + s] = acc[j];
  }
}

// ---------------------------------------------------------------- host linear algebra (b x b)
// Cholesky G = R^T R (upper R, row-major); false if a pivot is not positive
bool cholesky_upper(std::vector<double>& G, int b) {
  for (int j = 0; j < b; ++j) {
    double d = G[(size_t)j * b + j];
    for (int k = 0; k < j; ++k) d -= G[(size_t)k * b + j] * G[(size_t)k * b + j];
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double r = std::sqrt(d);
    G[(size_t)j * b + j] = r;
    for (int i = j + 1; i < b; ++i) {
      double v = G[(size_t)j * b + i];
      for (int k = 0; k < j; ++k) v -= G[(size_t)k * b + j] * G[(size_t)k * b + i];
      G[(size_t)j * b + i] = v / r;
    }
    for (int i = 0; i < j; ++i) G[(size_t)j * b + i] = 0.0;
  }
  return true;
}

// inverse of an upper triangular R (row-major), in place
void invert_upper(std::vector<double>& R, int b) {
  std::vector<double> Ri((size_t)b * b, 0.0);
  for (int j = 0; j < b; ++j) {
    Ri[(size_t)j * b + j] = 1.0 / R[(size_t)j * b + j];
    for (int i = j - 1; i >= 0; --i) {
      double v = 0.0;
      for (int k = i + 1; k <= j; ++k) v += R[(size_t)i * b + k] * Ri[(size_t)k * b + j];
      Ri[(size_t)i * b + j] = -v / R[(size_t)i * b + i];
    }
  }
  R.swap(Ri);
}

// cyclic Jacobi: H = W diag(theta) W^T for symmetric H (row-major); theta ascending, W columns
void jacobi_eigh(std::vector<double> H, int b, std::vector<double>& theta, std::vector<double>& W) {
  W.assign((size_t)b * b, 0.0);
  for (int i = 0; i < b; ++i) W[(size_t)i * b + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) {
        const double v = H[(size_t)i * b + j] * H[(size_t)i * b + j];
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < b - 1; ++p)
      for (int q = p + 1; q < b; ++q) {
        const double apq = H[(size_t)p * b + q];
        if (apq == 0.0) continue;
        const double app = H[(size_t)p * b + p], aqq = H[(size_t)q * b + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < b; ++k) {   // columns p, q
          const double hkp = H[(size_t)k * b + p], hkq = H[(size_t)k * b + q];
          H[(size_t)k * b + p] = c * hkp - s * hkq;
          H[(size_t)k * b + q] = s * hkp + c * hkq;
        }
        for (int k = 0; k < b; ++k) {   // rows p, q
          const double hpk = H[(size_t)p * b + k], hqk = H[(size_t)q * b + k];
          H[(size_t)p * b + k] = c * hpk - s * hqk;
          H[(size_t)q * b + k] = s * hpk + c * hqk;
        }
        for (int k = 0; k < b; ++k) {
          const double wkp = W[(size_t)k * b + p], wkq = W[(size_t)k * b + q];
          W[(size_t)k * b + p] = c * wkp - s * wkq;
          W[(size_t)k * b + q] = s * wkp + c * wkq;
        }
      }
  }
  std::vector<int> order(b);
  for (int i = 0; i < b; ++i) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int c) { return H[(size_t)a * b + a] < H[(size_t)c * b + c]; });
  theta.resize(b);
  std::vector<double> Ws((size_t)b * b);
  for (int j = 0; j < b; ++j) {
    theta[j] = H[(size_t)order[j] * b + order[j]];
    for (int i = 0; i < b; ++i) Ws[(size_t)i * b + j] = W[(size_t)i * b + order[j]];
  }
  W.swap(Ws);
}

struct EigWork {
  hp_ctx* ctx;
  LatGeom g;
  int V, b;
  double *X, *Y, *Z, *part, *Gd, *Wd;
  int nbx, spb;

  hp_status gram(const double* A, const double* B, std::vector<double>& G) {
    const int nt = (b + GT - 1) / GT;
    {
      ProfScope ps(ctx, "k_eig_gram");
      k_eig_gram<<<dim3(nbx, nt * nt), 256, 0, ctx->stream>>>(A, B, V, b, spb, part);
    }
    HP_LAUNCH_CHECK();
    k_eig_gram_sum<<<std::max(1, std::min(1024, (b * b + 255) / 256)), 256, 0, ctx->stream>>>(part, nbx, b * b, Gd);
    HP_LAUNCH_CHECK();
    G.resize((size_t)b * b);
    HP_CUDA(cudaMemcpyAsync(G.data(), Gd, sizeof(double) * b * b, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    return HP_OK;
  }
  // out = in W (b x b, host), out != in
  hp_status rotate(const double* in, const std::vector<double>& W, double* out) {
    HP_CUDA(cudaMemcpyAsync(Wd, W.data(), sizeof(double) * b * b, cudaMemcpyHostToDevice, ctx->stream));
    {
      ProfScope ps(ctx, "k_eig_rotate");
      k_eig_rotate<<<dim3(blocks_for(ctx, V, 256), (b + CJ - 1) / CJ), 256, 0, ctx->stream>>>(in, Wd, V, b, out);
    }
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status lincomb(double* out, const double* P, const double* Q, const double* R, double a, double c, double e) {
    const long long n = (long long)V * b;
    k_eig_lincomb<<<blocks_for(ctx, n, 256), 256, 0, ctx->stream>>>(out, P, Q, R, a, c, e, n);
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // X <- orthonormal basis of span(X): one shifted Cholesky QR, then two plain ones (Y is scratch)
  hp_status orthonormalise() {
    std::vector<double> G;
    for (int pass = 0; pass < 3; ++pass) {
      HP_TRY(gram(X, X, G));
      if (pass == 0) {   // shift: keeps the factorisation defined for a nearly dependent block
        double nrm = 0.0;
        for (int i = 0; i < b; ++i) nrm = std::max(nrm, G[(size_t)i * b + i]);
        const double sh = 11.0 * ((double)V * b + (double)b * (b + 1)) * 2.220446049250313e-16 * nrm;
        for (int i = 0; i < b; ++i) G[(size_t)i * b + i] += sh;
      }
      if (!cholesky_upper(G, b)) {
        hp_set_error("hp_laplacian_eigs: the block lost rank (Cholesky QR failed)");
        return HP_ENOCONV;
      }
      invert_upper(G, b);
      HP_TRY(rotate(X, G, Y));
      std::swap(X, Y);
    }
    return HP_OK;
  }
};

}  // namespace

extern "C" hp_status hp_laplacian_eigs(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                       double tol, int32_t max_sweeps, double* evecs, double* evals,
                                       double* resid) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 4, &dims));
  if (!op || op->kind != HP_OP_LAPLACIAN) {
    hp_set_error("hp_laplacian_eigs: the (real symmetric) Laplacian operator is required");
    return HP_EINVAL;
  }
  if (!std::isfinite(op->mass)) {
    hp_set_error("hp_laplacian_eigs: mass not finite");
    return HP_EINVAL;
  }
  LatticeSetup* ls = nullptr;
  HP_TRY(hp_get_lattice(ctx, dims, &ls));
  LatGeom g = ls->g;
  g.nd = 4;
  for (int j = (int)dims.size(); j < 8; ++j) g.L[j] = 1;
  g.op_kind = HP_OP_LAPLACIAN;
  const int V = g.V;
  if (k < 1 || 2LL * k > V || !(tol > 0.0) || !evecs || !evals) {
    hp_set_error("hp_laplacian_eigs: k in [1, V/2], tol > 0 and output arrays required");
    return HP_EINVAL;
  }
  HP_TRY(hp_prepare_mass(ctx, op, &g, "eigs"));
  // spectrum bound: the diagonal plus the 2 d hops of size 1 (Gershgorin)
  double mu_min = 0.0, mu_max = 0.0;
  if (op->mass_field) {
    std::vector<double> mf((size_t)V);
    HP_CUDA(cudaMemcpyAsync(mf.data(), g.mass_field, sizeof(double) * V, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    mu_min = *std::min_element(mf.begin(), mf.end());
    mu_max = *std::max_element(mf.begin(), mf.end());
  }
  const double l_max = 16.0 + op->mass + mu_max, l_low = op->mass + mu_min;
  const int b = std::min(V, k + std::max(8, k / 2));
  const int m = 12;   // degree of the filter per sweep
  EigWork w;
  w.ctx = ctx;
  w.g = g;
  w.V = V;
  w.b = b;
  w.nbx = (int)std::max<long long>(1, std::min<long long>(256, ((long long)V + 4095) / 4096));
  w.spb = (int)(((long long)V + w.nbx - 1) / w.nbx);
  const size_t blk = sizeof(double) * (size_t)V * b;
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "eigs.X", blk, &p));
  w.X = (double*)p;
  HP_TRY(hp_ws(ctx, "eigs.Y", blk, &p));
  w.Y = (double*)p;
  HP_TRY(hp_ws(ctx, "eigs.Z", blk, &p));
  w.Z = (double*)p;
  HP_TRY(hp_ws(ctx, "eigs.part", sizeof(double) * (size_t)w.nbx * b * b, &p));
  w.part = (double*)p;
  HP_TRY(hp_ws(ctx, "eigs.G", sizeof(double) * (size_t)b * b, &p));
  w.Gd = (double*)p;
  HP_TRY(hp_ws(ctx, "eigs.W", sizeof(double) * (size_t)b * b, &p));
  w.Wd = (double*)p;
  k_eig_fill<<<blocks_for(ctx, (long long)V * b, 256), 256, 0, ctx->stream>>>(w.X, (long long)V * b, 0x5eedULL + k);
  HP_LAUNCH_CHECK();
  HP_TRY(w.orthonormalise());
  std::vector<double> theta, W, H, rn(k, 0.0);
  const int sweeps = max_sweeps > 0 ? max_sweeps : 200;
  bool converged = false;
  for (int it = 0; it <= sweeps; ++it) {
    // Rayleigh-Ritz on the orthonormal block X: H = X^T A X, X <- X W, AX <- (A X) W
    HP_TRY(hp_apply_laplace(ctx, g, b, w.X, w.Z));
    HP_TRY(w.gram(w.X, w.Z, H));
    for (int i = 0; i < b; ++i)   // symmetrise the rounding
      for (int j = i + 1; j < b; ++j) H[(size_t)i * b + j] = H[(size_t)j * b + i] = 0.5 * (H[(size_t)i * b + j] + H[(size_t)j * b + i]);
    jacobi_eigh(H, b, theta, W);
    HP_TRY(w.rotate(w.X, W, w.Y));
    std::swap(w.X, w.Y);
    HP_TRY(w.rotate(w.Z, W, w.Y));   // A X in the rotated basis
    // residuals of the wanted pairs: R = A X - X diag(theta), ||R_j||^2 from the Gram of R with itself
    {
      std::vector<double> th(b);
      for (int j = 0; j < b; ++j) th[j] = theta[j];
      std::vector<double> D((size_t)b * b, 0.0);
      for (int j = 0; j < b; ++j) D[(size_t)j * b + j] = -th[j];
      HP_TRY(w.rotate(w.X, D, w.Z));                                   // Z = -X diag(theta)
      HP_TRY(w.lincomb(w.Z, w.Y, w.Z, nullptr, 1.0, 1.0, 0.0));        // Z = A X - X diag(theta)
      std::vector<double> RR;
      HP_TRY(w.gram(w.Z, w.Z, RR));
      converged = true;
      for (int j = 0; j < k; ++j) {
        rn[j] = std::sqrt(std::max(0.0, RR[(size_t)j * b + j])) / std::max(std::fabs(theta[j]), 1e-300);
        if (!(rn[j] <= tol)) converged = false;
      }
    }
    if (converged || it == sweeps) break;
    // Chebyshev filter of degree m damping [theta_b, l_max]; scaled at the lower bound l_low
    const double a = theta[b - 1], c0 = 0.5 * (l_max + a), e = 0.5 * (l_max - a);
    double sigma = e / (l_low - c0);
    const double tau = 2.0 / sigma;
    // Y = (A X - c0 X) sigma / e
    HP_TRY(hp_apply_laplace(ctx, g, b, w.X, w.Y));
    HP_TRY(w.lincomb(w.Y, w.Y, w.X, nullptr, sigma / e, -c0 * sigma / e, 0.0));
    for (int i = 2; i <= m; ++i) {
      const double sigma1 = 1.0 / (tau - sigma);
      // Z = 2 sigma1 / e (A Y - c0 Y) - sigma sigma1 X
      HP_TRY(hp_apply_laplace(ctx, g, b, w.Y, w.Z));
      HP_TRY(w.lincomb(w.Z, w.Z, w.Y, w.X, 2.0 * sigma1 / e, -2.0 * sigma1 * c0 / e, -sigma * sigma1));
      std::swap(w.X, w.Y);   // X <- Y
      std::swap(w.Y, w.Z);   // Y <- Z
      sigma = sigma1;
    }
    std::swap(w.X, w.Y);     // the filtered block
    HP_TRY(w.orthonormalise());
  }
  // outputs: the k lowest pairs
  const size_t out_bytes = sizeof(double) * (size_t)k * V;
  HP_CUDA(cudaMemcpyAsync(evecs, w.X, out_bytes, cudaMemcpyDefault, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < k; ++j) {
    evals[j] = theta[j];
    if (resid) resid[j] = rn[j];
  }
  if (!converged) {
    hp_set_error("hp_laplacian_eigs: %d sweeps without reaching tol", sweeps);
    return HP_ENOCONV;
  }
  return HP_OK;
}
