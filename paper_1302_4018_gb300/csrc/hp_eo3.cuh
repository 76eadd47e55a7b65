// Even-site hop of the even-odd iteration on the tensor cores (binary16 spinors and links, FP32
// accumulation): mid = A_e^-1 hop(in_o) for up to 32 right-hand sides of one lattice.
//
// For one site and one of the eight hops the Wilson term multiplies the 3x3 matrix Z (the link,
// or the adjoint of the backward link) by the two spin projections chi_h = psi_h + p_h psi_t(h),
// h = 0, 1, of the neighbour spinor psi of every right-hand side.  For a group of 8 right-hand
// sides that is one m16n8k16 MMA (mma.sync, binary16 x binary16 -> FP32):
//   rows    (rhs, h): 16
//   K       the real and imaginary parts of psi_h (pairs 0-2, colour b) and of psi_t(h)
//           (pairs 4-6): 12 of 16
//   columns (colour a, re / im) of Z chi_h: 6 of 8
//   B       [Z ; p Z] in the real form of the complex product
// so the tensor core forms the projection and the product in FP32 from the exact binary16
// inputs; the neighbour's per-site norm and the spin reconstruction act on the FP32 result.
// A lane (g, t) of the warp holds right-hand side g of the group and colour t (t = 3: the
// zero padding of K and of the columns), which is why binary16 fields keep the four spins of
// one colour in one 16-byte chunk: one load per lane gives its A fragment.
//
// tcgen05.mma takes its operands from shared memory in tiles of at least 64 rows sharing one B;
// here every site has its own B (its eight links), so the warp-level MMA with register operands
// is the form that fits.  Measured on GB300 it is slower than the FP32 pair kernels (the MMA
// covers one site and 8 right-hand sides, and the per-lane addressing, 16-byte scattered loads
// and FP32 reconstruction around it cost more instructions than the FMAs it replaces), so it is
// an opt-in variant (eo_kernel 6) that the autotuner does not time.
#pragma once

// D = A B with zero C (m16n8k16, row-major A, column-major B)
__device__ __forceinline__ void mma_m16n8k16(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                             unsigned b0, unsigned b1) {
  asm("mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %10, %10, %10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1), "f"(0.f));
}

// binary16 pairs (low half = real part): swap the halves; flip signs with XOR masks
__device__ __forceinline__ unsigned h2_swap(unsigned z) { return __byte_perm(z, 0u, 0x1032); }
constexpr unsigned H2_NEG_LO = 0x00008000u, H2_NEG_HI = 0x80000000u, H2_NEG = 0x80008000u;

// p z for the projection coefficient p in {1, -1, i, -i} (PC_ONE, PC_MONE, PC_I, PC_MI)
template <int CF>
__device__ __forceinline__ unsigned h2_times_coef(unsigned z) {
  if (CF == PC_ONE) return z;
  if (CF == PC_MONE) return z ^ H2_NEG;
  if (CF == PC_I) return h2_swap(z) ^ H2_NEG_LO;   // i (zr + i zi) = -zi + i zr
  return h2_swap(z) ^ H2_NEG_HI;                     // -i (zr + i zi) = zi - i zr
}
// the coefficients of (chi_re, chi_im) in the real (ri = 0) or imaginary (ri = 1) part of z chi
__device__ __forceinline__ unsigned h2_row(unsigned z, bool ri) { return ri ? h2_swap(z) : (z ^ H2_NEG_HI); }

template <int NG>
struct Eo3Acc {
  float v[NG][4][2];   // [group][spin][re, im] of colour t of right-hand side g
};

// one hop (direction MU, SIGN -1: forward neighbour with U_mu(x), +1: backward with U_mu(x - mu)^H)
// of the lane's site: nb the neighbour's half-site index, z the lane's link entry (binary16 pair,
// zero on padding lanes); the neighbour's spinor and norm of each running group are loaded here
template <int NG, int MU, int SIGN>
__device__ __forceinline__ void eo3_hop(const uint4* __restrict__ const (&pin)[NG], const float* __restrict__ const (&pn)[NG],
                                        const bool (&on)[NG], const bool (&any)[NG], bool colr, bool ri, int nb, unsigned z,
                                        float scale, Eo3Acc<NG>& acc) {
  constexpr int c0 = ProjCoef<MU, SIGN, 0>::coef, c1 = ProjCoef<MU, SIGN, 1>::coef;
  constexpr int t0 = ProjCoef<MU, SIGN, 0>::t, t1 = ProjCoef<MU, SIGN, 1>::t;
  // the second row's coefficient is the first's or its negative: fold the sign into its A entry
  static_assert(c1 == c0 || (c0 ^ c1) == 1, "projection coefficients of the two rows");
  constexpr unsigned flip1 = c1 == c0 ? 0u : H2_NEG;
  if (SIGN > 0) z ^= H2_NEG_HI;   // conj(U[b][a])
  const unsigned b0 = h2_row(z, ri), b1 = h2_row(h2_times_coef<c0>(z), ri);
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    if (!any[j]) continue;   // warp-uniform: no right-hand side of the group runs
    uint4 p = make_uint4(0u, 0u, 0u, 0u);
    float n = 0.f;
    if (on[j]) {
      if (colr) p = __ldg(pin[j] + nb);
      n = __ldg(pn[j] + nb);
    }
    const unsigned w0 = t0 == 2 ? p.z : p.w, w1 = t1 == 2 ? p.z : p.w;
    float d[4];
    mma_m16n8k16(d, p.x, p.y, w0, w1 ^ flip1, b0, b1);
    // W0 = (d0, d1) = (Z chi_0)[t], W1 = (d2, d3) = (Z chi_1)[t]; the reconstruction of the lower
    // spins follows the same rules as the FP32 stencils
    const float sc = scale * n;
    float(&o)[4][2] = acc.v[j];
    o[0][0] = fmaf(sc, d[0], o[0][0]);
    o[0][1] = fmaf(sc, d[1], o[0][1]);
    o[1][0] = fmaf(sc, d[2], o[1][0]);
    o[1][1] = fmaf(sc, d[3], o[1][1]);
    const float s = SIGN < 0 ? -sc : sc;
    if (MU == 0) {   // spin 2 += i s W1, spin 3 += i s W0
      o[2][0] = fmaf(-s, d[3], o[2][0]);
      o[2][1] = fmaf(s, d[2], o[2][1]);
      o[3][0] = fmaf(-s, d[1], o[3][0]);
      o[3][1] = fmaf(s, d[0], o[3][1]);
    } else if (MU == 1) {   // spin 2 += s W1, spin 3 -= s W0
      o[2][0] = fmaf(s, d[2], o[2][0]);
      o[2][1] = fmaf(s, d[3], o[2][1]);
      o[3][0] = fmaf(-s, d[0], o[3][0]);
      o[3][1] = fmaf(-s, d[1], o[3][1]);
    } else if (MU == 2) {   // spin 2 += i s W0, spin 3 -= i s W1
      o[2][0] = fmaf(-s, d[1], o[2][0]);
      o[2][1] = fmaf(s, d[0], o[2][1]);
      o[3][0] = fmaf(s, d[3], o[3][0]);
      o[3][1] = fmaf(-s, d[2], o[3][1]);
    } else {   // spin 2 += s W0, spin 3 += s W1
      o[2][0] = fmaf(s, d[0], o[2][0]);
      o[2][1] = fmaf(s, d[1], o[2][1]);
      o[3][0] = fmaf(s, d[2], o[3][0]);
      o[3][1] = fmaf(s, d[3], o[3][1]);
    }
  }
}

// the lane's binary16 link entry of direction mu at full site ls: entry e = 3 row + column of the
// 18-real form (entries 0-7 in U16f, 8 in U16g)
__device__ __forceinline__ unsigned eo3_link(const LatGeom& g, int mu, int ls, int e) {
  const unsigned* p = e < 8 ? reinterpret_cast<const unsigned*>(g.U16f + ((size_t)mu * 2 + (e >> 2)) * g.V + ls) + (e & 3)
                            : g.U16g + (size_t)mu * g.V + ls;
  return __ldg(p);
}

// ---- the kernel: one warp per site (site pairs h, h + 1 back to back, so that the second half
// of every 32-byte sector the first site's loads bring in is used at once), warps striding over
// the pairs so that the grid sweeps the lattice as one front
template <int NG>
__global__ void __launch_bounds__(128, 4) k_eo3_even(WArgs a, FieldPtr in, FieldPtr mid, int nslots, int lat) {
  const LatGeom g = a.lats[lat];
  const int lane = threadIdx.x & 31, gq = lane >> 2, tq = lane & 3;
  const bool colr = tq < 3;          // the lane carries colour tq
  const bool ri = gq & 1;            // its B column is the real (0) or imaginary (1) part of colour gq / 2
  const bool lk = colr && gq < 6;    // it holds a link entry
  const int efw = 3 * (gq >> 1) + tq, ebw = 3 * tq + (gq >> 1);
  const int nsite = g.V >> 1;
  const int Vmax = a.Vmax;
  bool on[NG], any[NG];
  const uint4* pin[NG];
  const float* pn[NG];
  uint4* pout[NG];
  float* pon[NG];
#pragma unroll
  for (int j = 0; j < NG; ++j) {
    const int slot = 8 * j + gq;
    on[j] = slot < nslots && eo_mask(a.st + slot, MASK_RUN);
    any[j] = __any_sync(0xffffffffu, on[j]);
    const int sl = slot < nslots ? slot : 0;
    pin[j] = (const uint4*)in.p + ((size_t)sl * 3 + (colr ? tq : 0)) * Vmax;
    pn[j] = in.nrm + (size_t)sl * Vmax;
    pout[j] = (uint4*)mid.p + ((size_t)sl * 3 + (colr ? tq : 0)) * Vmax;
    pon[j] = mid.nrm + (size_t)sl * Vmax;
  }
  const int warp = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int nwarp = gridDim.x * (blockDim.x >> 5);
  const int npair = (nsite + 1) >> 1;
  for (int pr = warp; pr < npair; pr += nwarp) {
    // lanes 8 e + k (k < 8) find hop k of site 2 pr + e: its neighbour and link site
    int my_nb = 0, my_ls = 0;
    float my_inv = 0.f;
    {
      const int e = (lane >> 3) & 1, k = lane & 7, mu = k >> 1;
      const int h = min(2 * pr + e, nsite - 1);
      int x[4], st[4];
      const int site = eo_site(g, h, 0, x, st);
      // direction mu of this lane by selection (a dynamic index would move x, st and g to local memory)
      const int L = mu == 0 ? g.L[0] : mu == 1 ? g.L[1] : mu == 2 ? g.L[2] : g.L[3];
      const int xm = mu == 0 ? x[0] : mu == 1 ? x[1] : mu == 2 ? x[2] : x[3];
      const int sm = mu == 0 ? st[0] : mu == 1 ? st[1] : mu == 2 ? st[2] : st[3];
      const int fw = (xm + 1 == L) ? site - (L - 1) * sm : site + sm;
      const int bw = (xm == 0) ? site + (L - 1) * sm : site - sm;
      my_nb = ((k & 1) ? bw : fw) >> 1;
      my_ls = (k & 1) ? bw : site;
      my_inv = 1.0f / site_diag<float>(g, site);
    }
#pragma unroll 1
    for (int e = 0; e < 2; ++e) {
      const int h = 2 * pr + e;
      if (h >= nsite) break;
      const float inv = __shfl_sync(0xffffffffu, my_inv, 8 * e);
      Eo3Acc<NG> acc;
#pragma unroll
      for (int j = 0; j < NG; ++j)
#pragma unroll
        for (int s = 0; s < 4; ++s) acc.v[j][s][0] = acc.v[j][s][1] = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int nb = __shfl_sync(0xffffffffu, my_nb, 8 * e + k);
        const int ls = __shfl_sync(0xffffffffu, my_ls, 8 * e + k);
        const int mu = k >> 1;
        const unsigned z = lk ? eo3_link(g, mu, ls, (k & 1) ? ebw : efw) : 0u;
        switch (k) {
          case 0: eo3_hop<NG, 0, -1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 1: eo3_hop<NG, 0, 1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 2: eo3_hop<NG, 1, -1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 3: eo3_hop<NG, 1, 1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 4: eo3_hop<NG, 2, -1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 5: eo3_hop<NG, 2, 1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          case 6: eo3_hop<NG, 3, -1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
          default: eo3_hop<NG, 3, 1>(pin, pn, on, any, colr, ri, nb, z, inv, acc); break;
        }
      }
      // store: per-site norm = max |component| over the three colour lanes of the row
#pragma unroll
      for (int j = 0; j < NG; ++j) {
        if (!any[j]) continue;
        const float(&o)[4][2] = acc.v[j];
        float m = 0.f;
#pragma unroll
        for (int s = 0; s < 4; ++s) m = fmaxf(m, fmaxf(fabsf(o[s][0]), fabsf(o[s][1])));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 1));
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, 2));
        if (!on[j]) continue;
        const float r = m > 0.f ? 1.0f / m : 0.f;
        if (colr) {
          uint4 w;
          w.x = Half2Ops<PR16>::from_f2(o[0][0] * r, o[0][1] * r);
          w.y = Half2Ops<PR16>::from_f2(o[1][0] * r, o[1][1] * r);
          w.z = Half2Ops<PR16>::from_f2(o[2][0] * r, o[2][1] * r);
          w.w = Half2Ops<PR16>::from_f2(o[3][0] * r, o[3][1] * r);
          pout[j][h] = w;
        }
        if (tq == 0) pon[j][h] = m;
      }
    }
  }
}
