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
//
// The Wilson operator's counterpart (hp_wilson_eigs; its filter runs the FP32 stencil until the
// residuals fall below 1e-5 or stop falling, the FP64 one after) runs the same iteration on complex spinor
// blocks for Q = gamma_5 D, Hermitian by gamma_5-hermiticity: the filter and the first
// Rayleigh-Ritz step act on Q^2 = D^H D (positive semidefinite, the same eigenvectors; Q itself is
// indefinite, and its Ritz values on an unconverged block can fall anywhere), a second Rayleigh-Ritz
// step with Q inside the span of the k lowest Q^2 Ritz vectors gives the pairs with their signed
// eigenvalues, ordered by |lambda| (the singular values of D).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "hp_internal.h"

hp_status hp_apply_laplace(hp_ctx* ctx, LatGeom g, int nrhs, const double* in, double* out);
hp_status hp_apply_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, const double* in,
                          double* out);

namespace {

constexpr int GT = 32;          // Gram tile (GT x GT entries per block)
// the largest k: each Rayleigh-Ritz step diagonalises a b x b matrix (b <= 2k + 8) on the host by
// cyclic Jacobi, O(b^3) per sweep, and the Gram launches take (b / GT)^2 blocks in grid y
#define HP_EIGS_MAX_K 1024
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

// ---------------------------------------------------------------- complex blocks (gamma_5 D)
constexpr int ZCH = 16;         // complex entries per shared-memory chunk of the complex Gram
constexpr int ZJ = 8;           // outputs per thread of the complex block rotation
typedef std::complex<double> zd;

__device__ __forceinline__ double2 zacc_conj(double2 x, double2 y, double2 acc) {   // acc + conj(x) y
  acc.x = fma(x.x, y.x, acc.x);
  acc.x = fma(x.y, y.y, acc.x);
  acc.y = fma(x.x, y.y, acc.y);
  acc.y = fma(-x.y, y.x, acc.y);
  return acc;
}
__device__ __forceinline__ double2 zacc(double2 x, double2 w, double2 acc) {   // acc + x w
  acc.x = fma(x.x, w.x, acc.x);
  acc.x = fma(-x.y, w.y, acc.x);
  acc.y = fma(x.x, w.y, acc.y);
  acc.y = fma(x.y, w.x, acc.y);
  return acc;
}

// partial complex Gram matrices: part[bx][i][j] = sum over the entries of chunk bx of conj(X[i][e]) Y[j][e]
// (vectors of n complex entries); 16 x 16 threads, 2 x 2 entries each
__global__ void __launch_bounds__(256) k_zeig_gram(const double2* __restrict__ X, const double2* __restrict__ Y,
                                                   long long n, int b, long long per_block, double2* __restrict__ part) {
  __shared__ double2 xs[GT][ZCH + 1], ys[GT][ZCH + 1];
  const int ntj = (b + GT - 1) / GT;
  const int i0 = (blockIdx.y / ntj) * GT, j0 = (blockIdx.y % ntj) * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double2 acc[2][2];
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) acc[u][v] = make_double2(0.0, 0.0);
  const long long e_begin = (long long)blockIdx.x * per_block;
  const long long e_end = std::min<long long>(n, e_begin + per_block);
  for (long long e0 = e_begin; e0 < e_end; e0 += ZCH) {
    for (int t = threadIdx.x; t < GT * ZCH; t += 256) {
      const int r = t / ZCH, c = t % ZCH;
      const long long e = e0 + c;
      xs[r][c] = (i0 + r < b && e < e_end) ? X[(size_t)(i0 + r) * n + e] : make_double2(0.0, 0.0);
      ys[r][c] = (j0 + r < b && e < e_end) ? Y[(size_t)(j0 + r) * n + e] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int c = 0; c < ZCH; ++c) {
      const double2 x0 = xs[2 * ty][c], x1 = xs[2 * ty + 1][c];
      const double2 y0 = ys[2 * tx][c], y1 = ys[2 * tx + 1][c];
      acc[0][0] = zacc_conj(x0, y0, acc[0][0]);
      acc[0][1] = zacc_conj(x0, y1, acc[0][1]);
      acc[1][0] = zacc_conj(x1, y0, acc[1][0]);
      acc[1][1] = zacc_conj(x1, y1, acc[1][1]);
    }
    __syncthreads();
  }
  double2* p = part + (size_t)blockIdx.x * b * b;
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + 2 * ty + u, j = j0 + 2 * tx + v;
      if (i < b && j < b) p[(size_t)i * b + j] = acc[u][v];
    }
}

// Z[j][e] = sum_i X[i][e] W[i][j] for the ZJ outputs j of blockIdx.y (W complex, row-major b x b)
__global__ void k_zeig_rotate(const double2* __restrict__ X, const double2* __restrict__ W, long long n, int b,
                              double2* __restrict__ Z) {
  const int j0 = blockIdx.y * ZJ;
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
    double2 acc[ZJ];
#pragma unroll
    for (int j = 0; j < ZJ; ++j) acc[j] = make_double2(0.0, 0.0);
    for (int i = 0; i < b; ++i) {
      const double2 x = X[(size_t)i * n + e];
      const double2* w = W + (size_t)i * b + j0;
#pragma unroll
      for (int j = 0; j < ZJ; ++j)
        if (j0 + j < b) acc[j] = zacc(x, __ldg(w + j), acc[j]);
    }
#pragma unroll
    for (int j = 0; j < ZJ; ++j)
      if (j0 + j < b) Z[(size_t)(j0 + j) * n + e] = acc[j];
  }
}

// X <- gamma_5 X on spinor fields [..][V][4][3]: gamma_5 = diag(1, 1, -1, -1) on the spins (chiral basis)
__global__ void k_gamma5(double2* __restrict__ X, long long total) {
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x)
    if ((t % 12) >= 6) X[t] = make_double2(-X[t].x, -X[t].y);
}

// out[j] = inv[j] gamma_5 Z[j] for the first k vectors (the left singular vectors u_j = D v_j / sigma_j
// from Z = Q X = gamma_5 D X)
__global__ void k_left_vectors(const double2* __restrict__ Z, const double* __restrict__ inv, long long n, int k,
                               double2* __restrict__ out) {
  const long long total = n * k;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long long)gridDim.x * blockDim.x) {
    const double s = inv[t / n] * ((t % 12) >= 6 ? -1.0 : 1.0);
    out[t] = make_double2(s * Z[t].x, s * Z[t].y);
  }
}

// residual norms: part[j][bx] = sum over the entries of chunk bx of |AX[j][e] - th[j] X[j][e]|^2 for
// the first k vectors (one block per chunk and vector; a fixed-order tree in shared memory)
__global__ void __launch_bounds__(256) k_zresid(const double2* __restrict__ AX, const double2* __restrict__ X,
                                                const double* __restrict__ th, long long n, int k, long long per_block,
                                                double* __restrict__ part) {
  __shared__ double sh[256];
  const long long e_begin = (long long)blockIdx.x * per_block;
  const long long e_end = std::min<long long>(n, e_begin + per_block);
  for (int j = blockIdx.y; j < k; j += gridDim.y) {
    const double t = th[j];
    const double2* a = AX + (size_t)j * n;
    const double2* x = X + (size_t)j * n;
    double acc = 0.0;
    for (long long e = e_begin + threadIdx.x; e < e_end; e += 256) {
      const double2 av = a[e], xv = x[e];
      const double rx = fma(-t, xv.x, av.x), ry = fma(-t, xv.y, av.y);
      acc = fma(rx, rx, acc);
      acc = fma(ry, ry, acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
      if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(size_t)j * gridDim.x + blockIdx.x] = sh[0];
    __syncthreads();
  }
}

// Cholesky G = R^H R of a Hermitian G (upper R, row-major); false if a pivot is not positive
bool cholesky_upper_z(std::vector<zd>& G, int b) {
  for (int j = 0; j < b; ++j) {
    double d = G[(size_t)j * b + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(G[(size_t)k * b + j]);
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    const double r = std::sqrt(d);
    G[(size_t)j * b + j] = r;
    for (int i = j + 1; i < b; ++i) {
      zd v = G[(size_t)j * b + i];
      for (int k = 0; k < j; ++k) v -= std::conj(G[(size_t)k * b + j]) * G[(size_t)k * b + i];
      G[(size_t)j * b + i] = v / r;
    }
    for (int i = 0; i < j; ++i) G[(size_t)j * b + i] = 0.0;
  }
  return true;
}

void invert_upper_z(std::vector<zd>& R, int b) {
  std::vector<zd> Ri((size_t)b * b, 0.0);
  for (int j = 0; j < b; ++j) {
    Ri[(size_t)j * b + j] = 1.0 / R[(size_t)j * b + j];
    for (int i = j - 1; i >= 0; --i) {
      zd v = 0.0;
      for (int k = i + 1; k <= j; ++k) v += R[(size_t)i * b + k] * Ri[(size_t)k * b + j];
      Ri[(size_t)i * b + j] = -v / R[(size_t)i * b + i];
    }
  }
  R.swap(Ri);
}

// cyclic Jacobi for a Hermitian H (row-major): H = W diag(theta) W^H, ordered by |theta|.  Each
// rotation first turns h_pq real (column q times e^{-i phi}, row q times e^{i phi}, phi = arg h_pq),
// then applies the real Jacobi rotation of the symmetric case.
void jacobi_eigh_z(std::vector<zd> H, int b, std::vector<double>& theta, std::vector<zd>& W) {
  W.assign((size_t)b * b, 0.0);
  for (int i = 0; i < b; ++i) W[(size_t)i * b + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < b; ++i)
      for (int j = 0; j < b; ++j) {
        const double v = std::norm(H[(size_t)i * b + j]);
        tot += v;
        if (i != j) off += v;
      }
    if (off <= 1e-30 * tot) break;
    for (int p = 0; p < b - 1; ++p)
      for (int q = p + 1; q < b; ++q) {
        const zd hpq = H[(size_t)p * b + q];
        const double apq = std::abs(hpq);
        if (apq == 0.0) continue;
        const zd ph = std::conj(hpq) / apq;   // e^{-i phi}
        for (int k = 0; k < b; ++k) {
          H[(size_t)k * b + q] *= ph;
          W[(size_t)k * b + q] *= ph;
        }
        for (int k = 0; k < b; ++k) H[(size_t)q * b + k] *= std::conj(ph);
        const double app = H[(size_t)p * b + p].real(), aqq = H[(size_t)q * b + q].real();
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < b; ++k) {   // columns p, q
          const zd hkp = H[(size_t)k * b + p], hkq = H[(size_t)k * b + q];
          H[(size_t)k * b + p] = c * hkp - s * hkq;
          H[(size_t)k * b + q] = s * hkp + c * hkq;
        }
        for (int k = 0; k < b; ++k) {   // rows p, q
          const zd hpk = H[(size_t)p * b + k], hqk = H[(size_t)q * b + k];
          H[(size_t)p * b + k] = c * hpk - s * hqk;
          H[(size_t)q * b + k] = s * hpk + c * hqk;
        }
        for (int k = 0; k < b; ++k) {
          const zd wkp = W[(size_t)k * b + p], wkq = W[(size_t)k * b + q];
          W[(size_t)k * b + p] = c * wkp - s * wkq;
          W[(size_t)k * b + q] = s * wkp + c * wkq;
        }
      }
  }
  std::vector<int> order(b);
  for (int i = 0; i < b; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int c) {
    return std::fabs(H[(size_t)a * b + a].real()) < std::fabs(H[(size_t)c * b + c].real());
  });
  theta.resize(b);
  std::vector<zd> Ws((size_t)b * b);
  for (int j = 0; j < b; ++j) {
    theta[j] = H[(size_t)order[j] * b + order[j]].real();
    for (int i = 0; i < b; ++i) Ws[(size_t)i * b + j] = W[(size_t)i * b + order[j]];
  }
  W.swap(Ws);
}

struct ZEigWork {
  hp_ctx* ctx;
  const hp_operator* op;
  LatGeom g;
  long long n;   // complex entries per vector (12 V)
  int b;
  double2 *X, *Y, *Z, *T, *part, *Gd, *Wd;
  int nbx;
  long long epb;
  int prec = HP_PREC_FP64;   // stencil precision of apply_q (the filter may run the FP32 one)

  // out = Q in = gamma_5 D in for the b vectors (FP64 or FP32 stencil, FP64 in and out)
  hp_status apply_q(const double2* in, double2* out) {
    HP_TRY(hp_apply_wilson(ctx, op, g, b, prec, (const double*)in, (double*)out));
    const long long tot = n * b;
    k_gamma5<<<blocks_for(ctx, tot, 256), 256, 0, ctx->stream>>>(out, tot);
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  hp_status apply_q2(const double2* in, double2* out) {   // out = Q^2 in (T scratch)
    HP_TRY(apply_q(in, T));
    return apply_q(T, out);
  }
  hp_status gram(const double2* A, const double2* B, std::vector<zd>& G) {
    const int nt = (b + GT - 1) / GT;
    {
      ProfScope ps(ctx, "k_zeig_gram");
      k_zeig_gram<<<dim3(nbx, nt * nt), 256, 0, ctx->stream>>>(A, B, n, b, epb, part);
    }
    HP_LAUNCH_CHECK();
    // the complex sum of the partials: the real kernel over both parts
    k_eig_gram_sum<<<std::max(1, std::min(1024, (2 * b * b + 255) / 256)), 256, 0, ctx->stream>>>(
        (const double*)part, nbx, 2 * b * b, (double*)Gd);
    HP_LAUNCH_CHECK();
    std::vector<double2> raw((size_t)b * b);
    HP_CUDA(cudaMemcpyAsync(raw.data(), Gd, sizeof(double2) * b * b, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    G.resize((size_t)b * b);
    for (size_t e = 0; e < G.size(); ++e) G[e] = zd(raw[e].x, raw[e].y);
    return HP_OK;
  }
  hp_status rotate(const double2* in, const std::vector<zd>& W, double2* out) {
    std::vector<double2> raw((size_t)b * b);
    for (size_t e = 0; e < raw.size(); ++e) raw[e] = make_double2(W[e].real(), W[e].imag());
    HP_CUDA(cudaMemcpyAsync(Wd, raw.data(), sizeof(double2) * b * b, cudaMemcpyHostToDevice, ctx->stream));
    {
      ProfScope ps(ctx, "k_zeig_rotate");
      k_zeig_rotate<<<dim3(blocks_for(ctx, n, 256), (b + ZJ - 1) / ZJ), 256, 0, ctx->stream>>>(in, Wd, n, b, out);
    }
    HP_LAUNCH_CHECK();
    HP_CUDA(cudaStreamSynchronize(ctx->stream));   // raw (host) must outlive the copy
    return HP_OK;
  }
  // out = a P + c Q + e R on the real and imaginary parts (real coefficients)
  hp_status lincomb(double2* out, const double2* P, const double2* Q, const double2* R, double a, double c, double e) {
    const long long m = 2 * n * b;
    k_eig_lincomb<<<blocks_for(ctx, m, 256), 256, 0, ctx->stream>>>((double*)out, (const double*)P, (const double*)Q,
                                                                     (const double*)R, a, c, e, m);
    HP_LAUNCH_CHECK();
    return HP_OK;
  }
  // r2[j] = ||AX_j - th_j X_j||^2 for j < k (th real); the partials summed on the host in chunk order
  hp_status resid_norms(const double2* AX, const double2* X, const std::vector<double>& th, int k,
                        std::vector<double>& r2) {
    HP_CUDA(cudaMemcpyAsync(Wd, th.data(), sizeof(double) * k, cudaMemcpyHostToDevice, ctx->stream));
    {
      ProfScope ps(ctx, "k_zresid");
      k_zresid<<<dim3(nbx, std::min(k, 65535)), 256, 0, ctx->stream>>>(AX, X, (const double*)Wd, n, k, epb,
                                                                        (double*)part);
    }
    HP_LAUNCH_CHECK();
    std::vector<double> raw((size_t)nbx * k);
    HP_CUDA(cudaMemcpyAsync(raw.data(), part, sizeof(double) * raw.size(), cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));   // th and raw (host) outlive the copies
    r2.assign(k, 0.0);
    for (int j = 0; j < k; ++j)
      for (int bx = 0; bx < nbx; ++bx) r2[j] += raw[(size_t)j * nbx + bx];
    return HP_OK;
  }
  hp_status orthonormalise() {
    std::vector<zd> G;
    for (int pass = 0; pass < 3; ++pass) {
      HP_TRY(gram(X, X, G));
      if (pass == 0) {
        double nrm = 0.0;
        for (int i = 0; i < b; ++i) nrm = std::max(nrm, G[(size_t)i * b + i].real());
        const double sh = 11.0 * ((double)n * b + (double)b * (b + 1)) * 2.220446049250313e-16 * nrm;
        for (int i = 0; i < b; ++i) G[(size_t)i * b + i] += sh;
      }
      if (!cholesky_upper_z(G, b)) {
        hp_set_error("hp_wilson_eigs: the block lost rank (Cholesky QR failed)");
        return HP_ENOCONV;
      }
      invert_upper_z(G, b);
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
  if (k < 1 || 2LL * k > V || k > HP_EIGS_MAX_K || !(tol > 0.0) || !evecs || !evals) {
    hp_set_error("hp_laplacian_eigs: k in [1, min(V/2, %d)], tol > 0 and output arrays required", HP_EIGS_MAX_K);
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

// the eigenpairs of Q = gamma_5 D with the smallest |lambda| (svd = false: evecs, evals signed), or the
// smallest singular triplets D v = sigma u (svd = true: evecs = v, left = u, evals = sigma), from the
// same filtered block iteration
static hp_status wilson_block_eigs(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                                   int32_t max_sweeps, bool svd, double* evecs, double* left, double* evals,
                                   double* resid) {
  const char* fn = svd ? "hp_wilson_svd" : "hp_wilson_eigs";
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 4, &dims));
  if (!op || op->kind != HP_OP_WILSON || !op->links) {
    hp_set_error("%s: a Wilson operator with links is required", fn);
    return HP_EINVAL;
  }
  if (!std::isfinite(op->mass) || !std::isfinite(op->kappa) || !std::isfinite(op->csw)) {
    hp_set_error("%s: mass / kappa / csw not finite", fn);
    return HP_EINVAL;
  }
  LatticeSetup* ls = nullptr;
  HP_TRY(hp_get_lattice(ctx, dims, &ls));
  LatGeom g = ls->g;
  g.nd = 4;
  for (int j = (int)dims.size(); j < 8; ++j) g.L[j] = 1;
  g.op_kind = HP_OP_WILSON;
  g.dof = 12;
  const int V = g.V;
  const long long n = 12LL * V;
  if (k < 1 || 2LL * k > n || k > HP_EIGS_MAX_K || !(tol > 0.0) || !evecs || !evals || (svd && !left)) {
    hp_set_error("%s: k in [1, min(6 V, %d)], tol > 0 and output arrays required", fn, HP_EIGS_MAX_K);
    return HP_EINVAL;
  }
  // spectrum bound of Q^2 = D^H D: ||D|| <= |1 + m| + max |mu| + 16 kappa (eight hops of norm 2 kappa)
  // + 12 csw kappa (six clover planes, ||sigma F|| <= 2)
  double mu_abs = 0.0;
  if (op->mass_field) {
    LatGeom gm = g;
    HP_TRY(hp_prepare_mass(ctx, op, &gm, "zeigs"));
    std::vector<double> mf((size_t)V);
    HP_CUDA(cudaMemcpyAsync(mf.data(), gm.mass_field, sizeof(double) * V, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    for (double v : mf) mu_abs = std::max(mu_abs, std::fabs(v));
  }
  const double dnorm = std::fabs(1.0 + op->mass) + mu_abs + 16.0 * std::fabs(op->kappa) +
                       12.0 * std::fabs(op->csw * op->kappa);
  double l_max = dnorm * dnorm;
  const double l_low = 0.0;
  // guard vectors: the low spectrum of gamma_5 D is dense, and the k-th pair converges at the rate
  // set by the gap between the k-th and the (b+1)-th values of Q^2, so the block is twice k (with
  // k + 8 the k-th and b-th values of a 16^4 problem lay within 0.7% and the modes near k never
  // separated)
  const int b = (int)std::min<long long>(n, 2LL * k + 8);
  const int m = 16;
  ZEigWork w;
  w.ctx = ctx;
  w.op = op;
  w.g = g;
  w.n = n;
  w.b = b;
  w.nbx = (int)std::max<long long>(1, std::min<long long>(256, (n + 4095) / 4096));
  w.epb = (n + w.nbx - 1) / w.nbx;
  const size_t blk = sizeof(double2) * (size_t)n * b;
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "zeigs.X", blk, &p));
  w.X = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.Y", blk, &p));
  w.Y = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.Z", blk, &p));
  w.Z = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.T", blk, &p));
  w.T = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.part", sizeof(double2) * (size_t)w.nbx * b * b, &p));
  w.part = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.G", sizeof(double2) * (size_t)b * b, &p));
  w.Gd = (double2*)p;
  HP_TRY(hp_ws(ctx, "zeigs.W", sizeof(double2) * (size_t)b * b, &p));
  w.Wd = (double2*)p;
  {
    // the top of the spectrum of Q^2 for the filter: 24 Lanczos steps from one random vector, the
    // largest Ritz value plus the last off-diagonal element (the safeguard of Zhou and Saad's
    // filtered subspace iteration), capped by the norm bound above
    ZEigWork v = w;
    v.b = 1;
    v.prec = HP_PREC_MIXED_FP32;   // a bound with a 1% margin: FP32 rounding is far inside it
    double2 *prev = w.Y, *cur = w.X, *nxt = w.Z;
    k_eig_fill<<<blocks_for(ctx, 2 * n, 256), 256, 0, ctx->stream>>>((double*)cur, 2 * n, 0x1a2c05ULL);
    HP_LAUNCH_CHECK();
    HP_CUDA(cudaMemsetAsync(prev, 0, sizeof(double2) * (size_t)n, ctx->stream));
    std::vector<zd> G;
    HP_TRY(v.gram(cur, cur, G));
    HP_TRY(v.lincomb(cur, cur, cur, nullptr, 1.0 / std::sqrt(G[0].real()), 0.0, 0.0));
    std::vector<double> alpha, beta;
    double bprev = 0.0;
    for (int j = 0; j < 24; ++j) {
      HP_TRY(v.apply_q2(cur, nxt));
      HP_TRY(v.lincomb(nxt, nxt, prev, nullptr, 1.0, -bprev, 0.0));
      HP_TRY(v.gram(cur, nxt, G));
      const double al = G[0].real();
      HP_TRY(v.lincomb(nxt, nxt, cur, nullptr, 1.0, -al, 0.0));
      HP_TRY(v.gram(nxt, nxt, G));
      const double be = std::sqrt(std::max(0.0, G[0].real()));
      alpha.push_back(al);
      beta.push_back(be);
      if (!(be > 1e-12 * std::fabs(al))) break;
      HP_TRY(v.lincomb(nxt, nxt, nxt, nullptr, 1.0 / be, 0.0, 0.0));
      std::swap(prev, cur);   // prev <- v_j, cur <- v_{j+1}, nxt <- free
      std::swap(cur, nxt);
      bprev = be;
    }
    const int L = (int)alpha.size();
    std::vector<double> Tm((size_t)L * L, 0.0), tth, tW;
    for (int i = 0; i < L; ++i) {
      Tm[(size_t)i * L + i] = alpha[i];
      if (i + 1 < L) Tm[(size_t)i * L + i + 1] = Tm[(size_t)(i + 1) * L + i] = beta[i];
    }
    jacobi_eigh(Tm, L, tth, tW);
    l_max = std::min(l_max, 1.01 * (tth[L - 1] + beta[L - 1]));
  }
  k_eig_fill<<<blocks_for(ctx, 2 * n * b, 256), 256, 0, ctx->stream>>>((double*)w.X, 2 * n * b, 0x5eed5ULL + k);
  HP_LAUNCH_CHECK();
  HP_TRY(w.orthonormalise());
  std::vector<double> theta, rn(k, 0.0);
  std::vector<zd> W, H;
  const int sweeps = max_sweeps > 0 ? max_sweeps : 200;
  bool converged = false;
  double top2 = 0.0;   // the largest Rayleigh-Ritz value of Q^2 on the block (the filter's damping bound)
  // the filter only has to raise the wanted directions: while the pairs are far from converged the
  // FP32 stencil does (its rounding stays below what a sweep removes), the last decades take the FP64
  // one.  Where the FP32 rounding floor of the residual lies depends on the operator (clover, the
  // spread of the spectrum, the residual's scale), so the switch is latched both at a fixed level and
  // as soon as the worst residual stops falling (less than 10% per sweep once below 1e-2).
  bool fp64_filter = false;
  double prev_worst = HUGE_VAL;
  auto pick_filter_precision = [&](double worst) {
    if (worst <= std::max(1e-5, 100.0 * tol) || (worst < 1e-2 && worst > 0.9 * prev_worst)) fp64_filter = true;
    prev_worst = worst;
    return fp64_filter ? HP_PREC_FP64 : HP_PREC_MIXED_FP32;
  };
  for (int it = 0; it <= sweeps; ++it) {
    // Rayleigh-Ritz with Q^2 = (Q X)^H (Q X) on the orthonormal block: the subspace and its order
    // (Q is indefinite, so its own Ritz values on a block mixing both ends of the spectrum can fall
    // anywhere, near 0 included; those of Q^2 are bounded by its spectrum); always the FP64 stencil
    w.prec = HP_PREC_FP64;
    HP_TRY(w.apply_q(w.X, w.Z));
    HP_TRY(w.gram(w.Z, w.Z, H));
    for (int i = 0; i < b; ++i) {   // Hermitian part (the rounding)
      H[(size_t)i * b + i] = H[(size_t)i * b + i].real();
      for (int j = i + 1; j < b; ++j) {
        const zd v = 0.5 * (H[(size_t)i * b + j] + std::conj(H[(size_t)j * b + i]));
        H[(size_t)i * b + j] = v;
        H[(size_t)j * b + i] = std::conj(v);
      }
    }
    std::vector<double> theta2;
    jacobi_eigh_z(H, b, theta2, W);   // ascending (theta2 >= 0)
    top2 = *std::max_element(theta2.begin(), theta2.end());
    HP_TRY(w.rotate(w.X, W, w.Y));
    std::swap(w.X, w.Y);
    HP_TRY(w.rotate(w.Z, W, w.Y));
    std::swap(w.Z, w.Y);             // Z = Q X in the rotated basis
    if (svd) {
      // singular triplets: the Q^2 Ritz pairs themselves, v_j = X_j, sigma_j = sqrt(theta2_j);
      // residual ||Q^2 v_j - sigma_j^2 v_j|| / sigma_j^2, Y = Q^2 X (FP64) serving the filter as well
      HP_TRY(w.apply_q(w.Z, w.Y));
      std::vector<double> r2;
      HP_TRY(w.resid_norms(w.Y, w.X, theta2, k, r2));
      converged = true;
      theta.assign(k, 0.0);
      for (int j = 0; j < k; ++j) {
        theta[j] = std::sqrt(std::max(0.0, theta2[j]));
        rn[j] = std::sqrt(std::max(0.0, r2[j])) / std::max(theta2[j], 1e-300);
        if (!(rn[j] <= tol)) converged = false;
      }
      if (converged || it == sweeps) break;
      w.prec = pick_filter_precision(*std::max_element(rn.begin(), rn.end()));
      const double a = std::min(top2, 0.99 * l_max);
      const double c0 = 0.5 * (l_max + a), e = 0.5 * (l_max - a);
      double sigma = e / (l_low - c0);
      const double tau = 2.0 / sigma;
      HP_TRY(w.lincomb(w.Y, w.Y, w.X, nullptr, sigma / e, -c0 * sigma / e, 0.0));   // Y = Q^2 X from above
      for (int i = 2; i <= m; ++i) {
        const double sigma1 = 1.0 / (tau - sigma);
        HP_TRY(w.apply_q2(w.Y, w.Z));
        HP_TRY(w.lincomb(w.Z, w.Z, w.Y, w.X, 2.0 * sigma1 / e, -2.0 * sigma1 * c0 / e, -sigma * sigma1));
        std::swap(w.X, w.Y);
        std::swap(w.Y, w.Z);
        sigma = sigma1;
      }
      std::swap(w.X, w.Y);
      HP_TRY(w.orthonormalise());
      continue;
    }
    // the eigenpairs of Q inside the span of the k lowest Q^2 Ritz vectors: Rayleigh-Ritz with Q there
    HP_TRY(w.gram(w.X, w.Z, H));
    std::vector<zd> Hk((size_t)k * k), W1;
    for (int i = 0; i < k; ++i) {
      Hk[(size_t)i * k + i] = H[(size_t)i * b + i].real();
      for (int j = i + 1; j < k; ++j) {
        const zd v = 0.5 * (H[(size_t)i * b + j] + std::conj(H[(size_t)j * b + i]));
        Hk[(size_t)i * k + j] = v;
        Hk[(size_t)j * k + i] = std::conj(v);
      }
    }
    jacobi_eigh_z(Hk, k, theta, W1);   // ordered by |theta|
    std::vector<zd> Wb((size_t)b * b, 0.0);
    for (int i = 0; i < b; ++i) Wb[(size_t)i * b + i] = 1.0;
    for (int i = 0; i < k; ++i)
      for (int j = 0; j < k; ++j) Wb[(size_t)i * b + j] = W1[(size_t)i * k + j];
    HP_TRY(w.rotate(w.X, Wb, w.Y));
    std::swap(w.X, w.Y);
    HP_TRY(w.rotate(w.Z, Wb, w.Y));   // Y = Q X, its first k columns the pairs' Q w_j
    {
      std::vector<double> r2;                                           // ||Q w_j - theta_j w_j||^2
      HP_TRY(w.resid_norms(w.Y, w.X, theta, k, r2));
      converged = true;
      for (int j = 0; j < k; ++j) {
        rn[j] = std::sqrt(std::max(0.0, r2[j])) / std::max(std::fabs(theta[j]), 1e-300);
        if (!(rn[j] <= tol)) converged = false;
      }
    }
    if (converged || it == sweeps) break;
    w.prec = pick_filter_precision(*std::max_element(rn.begin(), rn.end()));
    // Chebyshev filter of degree m on Q^2 damping [largest Q^2 Ritz value of the block, l_max], scaled at 0
    const double a = std::min(top2, 0.99 * l_max);
    const double c0 = 0.5 * (l_max + a), e = 0.5 * (l_max - a);
    double sigma = e / (l_low - c0);
    const double tau = 2.0 / sigma;
    HP_TRY(w.apply_q2(w.X, w.Y));
    HP_TRY(w.lincomb(w.Y, w.Y, w.X, nullptr, sigma / e, -c0 * sigma / e, 0.0));
    for (int i = 2; i <= m; ++i) {
      const double sigma1 = 1.0 / (tau - sigma);
      HP_TRY(w.apply_q2(w.Y, w.Z));
      HP_TRY(w.lincomb(w.Z, w.Z, w.Y, w.X, 2.0 * sigma1 / e, -2.0 * sigma1 * c0 / e, -sigma * sigma1));
      std::swap(w.X, w.Y);
      std::swap(w.Y, w.Z);
      sigma = sigma1;
    }
    std::swap(w.X, w.Y);
    HP_TRY(w.orthonormalise());
  }
  HP_CUDA(cudaMemcpyAsync(evecs, w.X, sizeof(double2) * (size_t)k * n, cudaMemcpyDefault, ctx->stream));
  if (svd) {   // u_j = D v_j / sigma_j = gamma_5 (Q v_j) / sigma_j, Q X in Z
    std::vector<double> inv(k);
    for (int j = 0; j < k; ++j) inv[j] = theta[j] > 0.0 ? 1.0 / theta[j] : 0.0;
    double* invd = nullptr;
    HP_TRY(hp_ws(ctx, "zeigs.inv", sizeof(double) * (size_t)k, (void**)&invd));
    HP_CUDA(cudaMemcpyAsync(invd, inv.data(), sizeof(double) * k, cudaMemcpyHostToDevice, ctx->stream));
    k_left_vectors<<<blocks_for(ctx, n * k, 256), 256, 0, ctx->stream>>>(w.Z, invd, n, k, w.T);
    HP_LAUNCH_CHECK();
    HP_CUDA(cudaMemcpyAsync(left, w.T, sizeof(double2) * (size_t)k * n, cudaMemcpyDefault, ctx->stream));
  }
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int j = 0; j < k; ++j) {
    evals[j] = theta[j];
    if (resid) resid[j] = rn[j];
  }
  if (!converged) {
    hp_set_error("%s: %d sweeps without reaching tol", fn, sweeps);
    return HP_ENOCONV;
  }
  return HP_OK;
}

extern "C" hp_status hp_wilson_eigs(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                                    int32_t max_sweeps, double* evecs, double* evals, double* resid) {
  return wilson_block_eigs(ctx, op, lat, k, tol, max_sweeps, false, evecs, nullptr, evals, resid);
}

extern "C" hp_status hp_wilson_svd(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k, double tol,
                                   int32_t max_sweeps, double* right, double* left, double* sigma, double* resid) {
  return wilson_block_eigs(ctx, op, lat, k, tol, max_sweeps, true, right, left, sigma, resid);
}
