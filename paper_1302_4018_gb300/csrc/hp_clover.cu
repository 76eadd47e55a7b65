// The clover term of the Clover-Wilson operator.
//
// Section 5.3 computes Tr D^-1 for the Clover-Wilson discretisation (it names
// the Sheikholeslami-Wohlert form and gives no formula).  The standard
// clover-leaf form is used: on every site
//   A(x) = (1 + m + mu(x)) 1 + C(x),
//   C(x) = -csw kappa sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
//   sigma_{mu nu} = (i/2) [g_mu, g_nu],
//   F_{mu nu}(x) = traceless part of (Q_{mu nu}(x) - Q_{mu nu}(x)^H) / (8i),
// Q_{mu nu}(x) the sum of the four plaquettes of the mu-nu plane that start and
// end at x, each run mu-then-nu.  In the chiral basis (g_5 = diag(1, 1, -1, -1))
// every sigma_{mu nu} is block diagonal in the spin pairs (0, 1) and (2, 3):
//   sigma_{jk} = -eps_{jkl} diag(P_l, P_l)   (j, k, l spatial, P the Pauli matrices)
//   sigma_{k4} = diag(P_k, -P_k),
// so A(x) is two Hermitian 6x6 blocks, stored packed (hp_internal.h) with their
// inverses for the even-odd iteration.  They are computed in FP64 from the FP64
// links, rounded to FP32 and float-float copies, and kept until a 64-bit hash
// of the links and mass field, or the coefficients, change (the gauge field of
// a trace computation is fixed, so the build runs once, not once per call).
#include <cstring>

#include "hp_fields.cuh"

namespace {

struct M3 {
  double2 e[9];   // row-major 3x3
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cmulc(double2 a, double2 b) {   // a * conj(b)
  return make_double2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
__device__ __forceinline__ double2 cconj_mul(double2 a, double2 b) {   // conj(a) * b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__device__ M3 link(const LatGeom& g, int site, int mu) {
  M3 m;
#pragma unroll
  for (int k = 0; k < 9; ++k) m.e[k] = g.U64[((size_t)mu * 9 + k) * g.V + site];
  return m;
}

// a b, a b^H, a^H b
__device__ M3 mul(const M3& a, const M3& b) {
  M3 c;
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      double2 t = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const double2 p = cmul(a.e[3 * r + k], b.e[3 * k + s]);
        t.x += p.x;
        t.y += p.y;
      }
      c.e[3 * r + s] = t;
    }
  return c;
}
__device__ M3 mul_h(const M3& a, const M3& b) {
  M3 c;
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      double2 t = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const double2 p = cmulc(a.e[3 * r + k], b.e[3 * s + k]);
        t.x += p.x;
        t.y += p.y;
      }
      c.e[3 * r + s] = t;
    }
  return c;
}
__device__ M3 h_mul(const M3& a, const M3& b) {
  M3 c;
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      double2 t = make_double2(0.0, 0.0);
      for (int k = 0; k < 3; ++k) {
        const double2 p = cconj_mul(a.e[3 * k + r], b.e[3 * k + s]);
        t.x += p.x;
        t.y += p.y;
      }
      c.e[3 * r + s] = t;
    }
  return c;
}

// site reached from coordinates x by d[j] steps along each direction (periodic)
__device__ int site_at(const LatGeom& g, const int (&x)[4], int mu, int dm, int nu, int dn) {
  int s = 0, stride = 1;
  for (int j = 0; j < 4; ++j) {
    int c = x[j] + (j == mu ? dm : 0) + (j == nu ? dn : 0);
    c = (c % g.L[j] + g.L[j]) % g.L[j];
    s += c * stride;
    stride *= g.L[j];
  }
  return s;
}

// F_{mu nu}(x) from the four leaves
__device__ M3 field_strength(const LatGeom& g, int site, const int (&x)[4], int mu, int nu) {
  const int xpm = site_at(g, x, mu, 1, nu, 0), xpn = site_at(g, x, mu, 0, nu, 1);
  const int xmm = site_at(g, x, mu, -1, nu, 0), xmn = site_at(g, x, mu, 0, nu, -1);
  const int xmmpn = site_at(g, x, mu, -1, nu, 1), xmmmn = site_at(g, x, mu, -1, nu, -1);
  const int xmnpm = site_at(g, x, mu, 1, nu, -1);
  // x -> x+mu -> x+mu+nu -> x+nu -> x
  M3 q = mul_h(mul_h(mul(link(g, site, mu), link(g, xpm, nu)), link(g, xpn, mu)), link(g, site, nu));
  // x -> x+nu -> x+nu-mu -> x-mu -> x
  M3 t = mul(mul_h(mul_h(link(g, site, nu), link(g, xmmpn, mu)), link(g, xmm, nu)), link(g, xmm, mu));
  for (int k = 0; k < 9; ++k) {
    q.e[k].x += t.e[k].x;
    q.e[k].y += t.e[k].y;
  }
  // x -> x-mu -> x-mu-nu -> x-nu -> x:  U_mu(x-mu)^H U_nu(x-mu-nu)^H = (U_nu(x-mu-nu) U_mu(x-mu))^H
  t = mul(h_mul(mul(link(g, xmmmn, nu), link(g, xmm, mu)), link(g, xmmmn, mu)), link(g, xmn, nu));
  for (int k = 0; k < 9; ++k) {
    q.e[k].x += t.e[k].x;
    q.e[k].y += t.e[k].y;
  }
  // x -> x-nu -> x-nu+mu -> x+mu -> x
  t = mul_h(mul(h_mul(link(g, xmn, nu), link(g, xmn, mu)), link(g, xmnpm, nu)), link(g, site, mu));
  for (int k = 0; k < 9; ++k) {
    q.e[k].x += t.e[k].x;
    q.e[k].y += t.e[k].y;
  }
  // F = (Q - Q^H) / (8i) = -i (Q - Q^H) / 8, then the trace removed
  M3 f;
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      const double2 a = q.e[3 * r + s], b = q.e[3 * s + r];
      const double dx = a.x - b.x, dy = a.y + b.y;   // Q_rs - conj(Q_sr)
      f.e[3 * r + s] = make_double2(dy / 8.0, -dx / 8.0);
    }
  const double tr = (f.e[0].x + f.e[4].x + f.e[8].x) / 3.0;   // F Hermitian: real trace
  f.e[0].x -= tr;
  f.e[4].x -= tr;
  f.e[8].x -= tr;
  return f;
}

// spin factor (2x2, within one chirality block) of sigma_{mu nu}, pair p = (mu<nu) in the order
// (0,1) (0,2) (0,3) (1,2) (1,3) (2,3), block b = 0 (spins 0, 1) or 1 (spins 2, 3)
__device__ void spin_factor(int p, int b, double2 (&s)[4]) {
  // Pauli matrices P_0, P_1, P_2 (row-major 2x2)
  const double2 z = make_double2(0.0, 0.0), one = make_double2(1.0, 0.0), i1 = make_double2(0.0, 1.0);
  double2 P[3][4] = {{z, one, one, z},
                     {z, make_double2(0.0, -1.0), i1, z},
                     {one, z, z, make_double2(-1.0, 0.0)}};
  int l = 0;
  double sg = 1.0;
  switch (p) {
    case 0: l = 2; sg = -1.0; break;               // sigma_{12} = -diag(P_3, P_3)
    case 1: l = 1; sg = 1.0; break;                // sigma_{13} = +diag(P_2, P_2)
    case 2: l = 0; sg = b ? -1.0 : 1.0; break;     // sigma_{14} = diag(P_1, -P_1)
    case 3: l = 0; sg = -1.0; break;               // sigma_{23} = -diag(P_1, P_1)
    case 4: l = 1; sg = b ? -1.0 : 1.0; break;     // sigma_{24} = diag(P_2, -P_2)
    default: l = 2; sg = b ? -1.0 : 1.0; break;    // sigma_{34} = diag(P_3, -P_3)
  }
  for (int k = 0; k < 4; ++k) s[k] = make_double2(sg * P[l][k].x, sg * P[l][k].y);
}

// 6x6 complex inverse by Gauss-Jordan elimination with partial pivoting; false if singular
__device__ bool invert6(double2 (&a)[6][6], double2 (&inv)[6][6]) {
  for (int r = 0; r < 6; ++r)
    for (int c = 0; c < 6; ++c) inv[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  for (int col = 0; col < 6; ++col) {
    int piv = col;
    double best = a[col][col].x * a[col][col].x + a[col][col].y * a[col][col].y;
    for (int r = col + 1; r < 6; ++r) {
      const double m = a[r][col].x * a[r][col].x + a[r][col].y * a[r][col].y;
      if (m > best) {
        best = m;
        piv = r;
      }
    }
    if (!(best > 0.0)) return false;
    if (piv != col)
      for (int c = 0; c < 6; ++c) {
        double2 t = a[col][c];
        a[col][c] = a[piv][c];
        a[piv][c] = t;
        t = inv[col][c];
        inv[col][c] = inv[piv][c];
        inv[piv][c] = t;
      }
    const double2 p = a[col][col];
    const double pm = p.x * p.x + p.y * p.y;
    const double2 ip = make_double2(p.x / pm, -p.y / pm);
    for (int c = 0; c < 6; ++c) {
      a[col][c] = cmul(a[col][c], ip);
      inv[col][c] = cmul(inv[col][c], ip);
    }
    for (int r = 0; r < 6; ++r) {
      if (r == col) continue;
      const double2 f = a[r][col];
      for (int c = 0; c < 6; ++c) {
        const double2 u = cmul(f, a[col][c]), v = cmul(f, inv[col][c]);
        a[r][c].x -= u.x;
        a[r][c].y -= u.y;
        inv[r][c].x -= v.x;
        inv[r][c].y -= v.y;
      }
    }
  }
  return true;
}

// packed entry e (0..35) of a Hermitian 6x6 block: diagonal reals, then the upper entries
__device__ void pack6(const double2 (&m)[6][6], double (&out)[36]) {
  for (int i = 0; i < 6; ++i) out[i] = m[i][i].x;
  int k = 6;
  for (int i = 0; i < 6; ++i)
    for (int j = i + 1; j < 6; ++j) {
      out[k] = m[i][j].x;
      out[k + 1] = m[i][j].y;
      k += 2;
    }
}

// one thread per site: A(x) and A(x)^-1 in FP64; a singular block sets *err
__global__ void k_clover_build(LatGeom g, double csw, double2* __restrict__ A64, double2* __restrict__ Ai64,
                               int* __restrict__ err) {
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < g.V; site += gridDim.x * blockDim.x) {
    int x[4], st[4];
    site_coords(g, site, x, st);
    M3 F[6];
    int p = 0;
    for (int mu = 0; mu < 4; ++mu)
      for (int nu = mu + 1; nu < 4; ++nu) F[p++] = field_strength(g, site, x, mu, nu);
    const double d = 1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0);
    const double f = -csw * g.kappa;
    for (int b = 0; b < 2; ++b) {
      double2 a[6][6], ai[6][6];
      for (int r = 0; r < 6; ++r)
        for (int c = 0; c < 6; ++c) a[r][c] = make_double2(r == c ? d : 0.0, 0.0);
      for (int q = 0; q < 6; ++q) {
        double2 s[4];
        spin_factor(q, b, s);
        for (int si = 0; si < 2; ++si)
          for (int ti = 0; ti < 2; ++ti)
            for (int c = 0; c < 3; ++c)
              for (int e = 0; e < 3; ++e) {
                const double2 v = cmul(s[2 * si + ti], F[q].e[3 * c + e]);
                a[3 * si + c][3 * ti + e].x += f * v.x;
                a[3 * si + c][3 * ti + e].y += f * v.y;
              }
      }
      double pa[36], pi[36];
      pack6(a, pa);
      if (!invert6(a, ai)) atomicExch(err, 1);
      pack6(ai, pi);
      for (int k = 0; k < 18; ++k) {
        A64[(size_t)(18 * b + k) * g.V + site] = make_double2(pa[2 * k], pa[2 * k + 1]);
        Ai64[(size_t)(18 * b + k) * g.V + site] = make_double2(pi[2 * k], pi[2 * k + 1]);
      }
    }
  }
}

// FP64 packed blocks -> FP32 high parts and FP32 low parts (float-float)
__global__ void k_clover_round(const double2* __restrict__ A64, int V, float4* __restrict__ hi,
                               float4* __restrict__ lo) {
  const long long total = 18LL * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(t / V), site = (int)(t - (long long)q * V);   // float4 chunk q
    const double2 u = A64[(size_t)(2 * q) * V + site], w = A64[(size_t)(2 * q + 1) * V + site];
    const double v[4] = {u.x, u.y, w.x, w.y};
    float h[4], l[4];
    for (int k = 0; k < 4; ++k) {
      h[k] = (float)v[k];
      l[k] = (float)(v[k] - (double)h[k]);
    }
    hi[t] = make_float4(h[0], h[1], h[2], h[3]);
    lo[t] = make_float4(l[0], l[1], l[2], l[3]);
  }
}

// position-dependent 64-bit hash of n words: sum over i of a SplitMix64-style mix of (word_i, i);
// equal inputs give equal sums in any summation order
__global__ void k_hash64(const unsigned long long* __restrict__ p, long long n, unsigned long long salt,
                         unsigned long long* __restrict__ out) {
  unsigned long long h = 0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = __ldg(p + i) ^ ((unsigned long long)(i + 1) * 0x9E3779B97F4A7C15ull) ^ salt;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    h += z ^ (z >> 31);
  }
  for (int o = 16; o > 0; o >>= 1) h += __shfl_down_sync(0xffffffffu, h, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, h);
}

}  // namespace

hp_status hp_prepare_clover(hp_ctx* ctx, const hp_operator* op, LatGeom* g, const char* tag) {
  g->clover = 0;
  g->A64 = g->Ai64 = nullptr;
  g->A32 = g->A32l = g->Ai32 = g->Ai32l = nullptr;
  if (op->kind != HP_OP_WILSON || op->csw == 0.0) return HP_OK;
  const size_t V = (size_t)g->V;
  const std::string base(tag);
  void *a64 = nullptr, *ai64 = nullptr, *a32 = nullptr, *a32l = nullptr, *ai32 = nullptr, *ai32l = nullptr,
       *err = nullptr;
  HP_TRY(hp_ws(ctx, (base + ".A64").c_str(), sizeof(double2) * 36 * V, &a64));
  HP_TRY(hp_ws(ctx, (base + ".Ai64").c_str(), sizeof(double2) * 36 * V, &ai64));
  HP_TRY(hp_ws(ctx, (base + ".A32").c_str(), sizeof(float4) * 18 * V, &a32));
  HP_TRY(hp_ws(ctx, (base + ".A32l").c_str(), sizeof(float4) * 18 * V, &a32l));
  HP_TRY(hp_ws(ctx, (base + ".Ai32").c_str(), sizeof(float4) * 18 * V, &ai32));
  HP_TRY(hp_ws(ctx, (base + ".Ai32l").c_str(), sizeof(float4) * 18 * V, &ai32l));
  HP_TRY(hp_ws(ctx, (base + ".Aerr").c_str(), sizeof(int), &err));
  // the inputs' hash: links (FP64 copy of the caller's array) and mass field
  void* hbuf = nullptr;
  HP_TRY(hp_ws(ctx, (base + ".Ahash").c_str(), sizeof(unsigned long long), &hbuf));
  HP_CUDA(cudaMemsetAsync(hbuf, 0, sizeof(unsigned long long), ctx->stream));
  k_hash64<<<blocks_for(ctx, 36LL * (long long)V, 256), 256, 0, ctx->stream>>>(
      (const unsigned long long*)g->U64, 72LL * (long long)V, 0x1ull, (unsigned long long*)hbuf);
  HP_LAUNCH_CHECK();
  if (g->mass_field) {
    k_hash64<<<blocks_for(ctx, (long long)V, 256), 256, 0, ctx->stream>>>(
        (const unsigned long long*)g->mass_field, (long long)V, 0x2ull, (unsigned long long*)hbuf);
    HP_LAUNCH_CHECK();
  }
  ctx->launches += g->mass_field ? 2 : 1;
  unsigned long long hash = 0;
  HP_CUDA(cudaMemcpyAsync(&hash, hbuf, sizeof(hash), cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  hp_ctx::CloverKey& key = ctx->clover_keys[base];
  const bool same = key.buf == a64 && key.hash == hash && key.csw == op->csw && key.kappa == op->kappa &&
                    key.mass == op->mass && key.V == (int)V && key.hash != 0;
  if (same) {
    g->clover = 1;
    g->A64 = (const double2*)a64;
    g->Ai64 = (const double2*)ai64;
    g->A32 = (const float4*)a32;
    g->A32l = (const float4*)a32l;
    g->Ai32 = (const float4*)ai32;
    g->Ai32l = (const float4*)ai32l;
    return HP_OK;
  }
  key.buf = nullptr;   // invalid until the rebuild below succeeds
  HP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  {
    ProfScope ps(ctx, "k_clover_build");
    k_clover_build<<<blocks_for(ctx, (long long)V, 128), 128, 0, ctx->stream>>>(*g, op->csw, (double2*)a64,
                                                                                 (double2*)ai64, (int*)err);
  }
  HP_LAUNCH_CHECK();
  {
    ProfScope ps(ctx, "k_clover_round");
    k_clover_round<<<blocks_for(ctx, 18LL * (long long)V, 256), 256, 0, ctx->stream>>>((const double2*)a64, (int)V,
                                                                                      (float4*)a32, (float4*)a32l);
    k_clover_round<<<blocks_for(ctx, 18LL * (long long)V, 256), 256, 0, ctx->stream>>>(
        (const double2*)ai64, (int)V, (float4*)ai32, (float4*)ai32l);
  }
  HP_LAUNCH_CHECK();
  int herr = 0;
  HP_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (herr) {
    hp_set_error("clover term: a diagonal block 1 + m + mu(x) + C(x) is singular");
    return HP_EINVAL;
  }
  key.hash = hash;
  key.csw = op->csw;
  key.kappa = op->kappa;
  key.mass = op->mass;
  key.V = (int)V;
  key.buf = a64;
  g->clover = 1;
  g->A64 = (const double2*)a64;
  g->Ai64 = (const double2*)ai64;
  g->A32 = (const float4*)a32;
  g->A32l = (const float4*)a32l;
  g->Ai32 = (const float4*)ai32;
  g->Ai32l = (const float4*)ai32l;
  return HP_OK;
}
