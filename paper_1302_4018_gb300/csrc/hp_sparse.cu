// Hierarchical probing of a general sparse matrix (Section 2.1, Algorithm 1;
// the probing basis of Section 2.2, Eq. Hperm-general-recursive).
//
// Algorithm 1 colours the graph of A greedily, and recurses into the rows of
// every colour with the block graph A(rows, :) A(:, rows) until a block is
// dense or fully disconnected.  Two facts make it data parallel:
//
// * the greedy colouring of a block visits its rows in increasing global
//   index (the recursion reorders rows by a stable sort on colour, so within
//   any block the order is the original one), and a greedy colouring in a
//   fixed order is what Jones-Plassmann rounds produce when the priority is
//   that order: a row takes the smallest colour none of its lower-indexed
//   neighbours has as soon as all of them are coloured.  Blocks of one level
//   share no edges, so one sweep colours every block of the level at once,
//   and the result is the sequential greedy colouring, bit for bit;
// * block identity needs no permutation: a block is named by the first
//   position its rows would take in perm, and a child block (parent b, colour
//   c) by the exclusive prefix sum of the per-(b, c) row counts, stored at
//   slot start(b) + c (a block of s rows has at most s colours, so the slots
//   of different blocks never collide).
//
// The next level's graph is built for the recursing rows only: the two-hop
// neighbours x of v (v -> w -> x in the current level graph) that fall in
// v's child block, deduplicated in a hash table private to v (twice the
// candidate count, linear probing), then compacted into CSR.  The output is
// every row's colour path paths[l][i] (colour at level l + 1, 0 below the
// level where its block stopped) and the colour count c(l) of each level.
//
// The probing vector m has the mixed-radix digits d_l(m) of m (level 1 least
// significant) and entry z_m(i) = prod_l exp(2 pi i d_l(m) paths[l][i] / c(l)).
// The trace runs the Laplacian CG engine with the CSR rows as the operator.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <vector>

#include "hp_internal.h"

namespace {

constexpr int ST = 256;   // threads per block of the colouring kernels

__global__ void k_sp_validate(int n, const int* __restrict__ rp, const int* __restrict__ ci, long long nnz,
                              int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    if (rp[i + 1] < rp[i]) atomicOr(bad, 1);
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += stride) {
    const int c = ci[e];
    if (c < 0 || c >= n) atomicOr(bad, 2);
  }
}

// level-1 graph: the pattern of A (diagonal and duplicate entries kept: they change no colour)
__global__ void k_sp_graph0(int n, const int* __restrict__ rp, long long* __restrict__ grp,
                            unsigned char* __restrict__ act, int* __restrict__ col, int* __restrict__ bstart) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += stride) {
    grp[i] = rp[i];
    if (i < n) {
      act[i] = 1;
      col[i] = -1;
      bstart[i] = 0;
    }
  }
}

// One Jones-Plassmann round with priority = row index: an uncoloured active row whose
// lower-indexed neighbours are all coloured takes the smallest colour none of them has.
// Colours are final once written, so reading a neighbour coloured earlier in the same
// round is as good as reading it in the next.  *pending counts rows left uncoloured.
__global__ void __launch_bounds__(ST) k_sp_jp(int n, const long long* __restrict__ rp, const int* __restrict__ ci,
                                              const unsigned char* __restrict__ act, int* col,
                                              unsigned int* __restrict__ pending) {
  volatile int* vcol = col;
  unsigned int left = 0;
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    if (!act[v] || vcol[v] >= 0) continue;
    const long long e0 = rp[v], e1 = rp[v + 1];
    unsigned long long used = 0;
    bool ready = true;
    for (long long e = e0; e < e1; ++e) {
      const int u = ci[e];
      if (u >= v) continue;
      const int c = vcol[u];
      if (c < 0) {
        ready = false;
        break;
      }
      if (c < 64) used |= 1ull << c;
    }
    if (!ready) {
      ++left;
      continue;
    }
    int c = 0;
    if (~used) {
      c = __ffsll((long long)~used) - 1;
    } else {   // the first 64 colours are taken: scan the next windows of 64
      for (int base = 64;; base += 64) {
        unsigned long long w = 0;
        for (long long e = e0; e < e1; ++e) {
          const int u = ci[e];
          if (u >= v) continue;
          const int d = vcol[u] - base;
          if (d >= 0 && d < 64) w |= 1ull << d;
        }
        if (~w) {
          c = base + __ffsll((long long)~w) - 1;
          break;
        }
      }
    }
    vcol[v] = c;
  }
  for (int o = 16; o > 0; o >>= 1) left += __shfl_down_sync(0xffffffffu, left, o);
  if ((threadIdx.x & 31) == 0 && left) atomicAdd(pending, left);
}

// Per-block colour counts (greedy colours are 0 .. k-1, so the count is the largest + 1),
// the level's largest count, and the colour paths of the level.  Warp lanes of one block
// combine their maxima before the atomic.
__global__ void __launch_bounds__(ST) k_sp_stats(int n, const unsigned char* __restrict__ act,
                                                 const int* __restrict__ col, const int* __restrict__ bstart,
                                                 int* __restrict__ bncol, int* __restrict__ radix,
                                                 int* __restrict__ path_l) {
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  int lvl_max = 0;
  for (int v0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
    const int v = v0 + lane;
    const bool ok = v < n && act[v];
    const int key = ok ? bstart[v] : -1;
    const int val = ok ? col[v] + 1 : 0;
    if (ok) path_l[v] = col[v];
    lvl_max = max(lvl_max, val);
    const unsigned int grp = __match_any_sync(0xffffffffu, key);
    const int gmax = __reduce_max_sync(grp, val);
    if (ok && lane == __ffs(grp) - 1) atomicMax(bncol + key, gmax);
  }
  lvl_max = __reduce_max_sync(0xffffffffu, lvl_max);
  if (lane == 0 && lvl_max) atomicMax(radix, lvl_max);
}

// Whether each row's block recurses (neither dense nor one colour, and levels remain), and
// the row counts of the child blocks at slot start(b) + colour; rows of stopped blocks count
// at their block's start so that the prefix sum keeps every block's range.
__global__ void __launch_bounds__(ST) k_sp_count(int n, const unsigned char* __restrict__ act,
                                                 const int* __restrict__ col, const int* __restrict__ bstart,
                                                 const int* __restrict__ bsize, const int* __restrict__ bncol,
                                                 int last_level, unsigned char* __restrict__ rec,
                                                 int* __restrict__ cnt, int* __restrict__ any_rec) {
  const int lane = threadIdx.x & 31;
  const int stride = gridDim.x * blockDim.x;
  int any = 0;
  for (int v0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); v0 < n; v0 += stride) {
    const int v = v0 + lane;
    int key = -1;
    if (v < n) {
      const int b = bstart[v];
      bool r = false;
      if (act[v] && !last_level) {
        const int nc = bncol[b];
        r = nc != bsize[b] && nc != 1;
      }
      rec[v] = r ? 1 : 0;
      any |= r;
      key = b + (r ? col[v] : 0);
    }
    const unsigned int grp = __match_any_sync(0xffffffffu, key);
    if (key >= 0 && lane == __ffs(grp) - 1) atomicAdd(cnt + key, __popc(grp));
  }
  any = (int)__reduce_or_sync(0xffffffffu, (unsigned int)any);
  if (lane == 0 && any) atomicOr(any_rec, 1);
}

// child block starts and sizes; recursing rows become the next level's active, uncoloured rows
__global__ void k_sp_relabel(int n, const unsigned char* __restrict__ rec, int* __restrict__ col,
                             const int* __restrict__ bstart, const int* __restrict__ cnt, const int* __restrict__ S,
                             int* __restrict__ nbstart, int* __restrict__ nbsize, unsigned char* __restrict__ act) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const bool r = rec[v] != 0;
    const int slot = bstart[v] + (r ? col[v] : 0);
    const int s = S[slot];
    nbstart[v] = s;
    nbsize[s] = cnt[slot];
    act[v] = r ? 1 : 0;
    if (r) col[v] = -1;
  }
}

__device__ __forceinline__ unsigned int sp_hash(unsigned int x) {   // integer mixer (Murmur3 finaliser)
  x ^= x >> 16;
  x *= 0x85ebca6bu;
  x ^= x >> 13;
  x *= 0xc2b2ae35u;
  x ^= x >> 16;
  return x;
}

// two-hop candidates of each recursing row inside its child block -> hash table size
__global__ void __launch_bounds__(ST) k_sp_hcount(int n, const long long* __restrict__ rp, const int* __restrict__ ci,
                                                  const unsigned char* __restrict__ act,
                                                  const int* __restrict__ nb, long long* __restrict__ hsz) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    long long cand = 0;
    if (act[v]) {
      const int bv = nb[v];
      for (long long e = rp[v]; e < rp[v + 1]; ++e) {
        const int w = ci[e];
        for (long long f = rp[w]; f < rp[w + 1]; ++f) cand += nb[ci[f]] == bv;
      }
    }
    long long h = 0;
    if (cand) {
      h = 1;
      while (h < 2 * cand) h <<= 1;
    }
    hsz[v] = h;
  }
}

__global__ void __launch_bounds__(ST) k_sp_hinsert(int n, const long long* __restrict__ rp,
                                                   const int* __restrict__ ci, const unsigned char* __restrict__ act,
                                                   const int* __restrict__ nb, const long long* __restrict__ hoff,
                                                   const long long* __restrict__ hsz, int* __restrict__ table,
                                                   long long* __restrict__ ucnt) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    long long u = 0;
    if (act[v] && hsz[v]) {
      int* t = table + hoff[v];
      const unsigned long long mask = (unsigned long long)hsz[v] - 1;
      const int bv = nb[v];
      for (long long e = rp[v]; e < rp[v + 1]; ++e) {
        const int w = ci[e];
        for (long long f = rp[w]; f < rp[w + 1]; ++f) {
          const int x = ci[f];
          if (nb[x] != bv) continue;
          unsigned long long h = sp_hash((unsigned int)x) & mask;
          while (true) {   // ends: the table has at least twice as many slots as candidates
            const int y = t[h];
            if (y == x) break;
            if (y < 0) {
              t[h] = x;
              ++u;
              break;
            }
            h = (h + 1) & mask;
          }
        }
      }
    }
    ucnt[v] = u;
  }
}

__global__ void __launch_bounds__(ST) k_sp_hwrite(int n, const long long* __restrict__ hoff,
                                                  const long long* __restrict__ hsz, const int* __restrict__ table,
                                                  const long long* __restrict__ nrp, int* __restrict__ nci) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int* t = table + hoff[v];
    long long o = nrp[v];
    for (long long h = 0; h < hsz[v]; ++h)
      if (t[h] >= 0) nci[o++] = t[h];
  }
}

// ------------------------------------------------------------ exclusive scan
// out[i] = sum_{j<i} in[i], out[n] = total; tiles of 1024 x 8 values, then one block over
// the tile sums (in chunks, carrying the running total), then the tile offsets.
constexpr int SC_T = 1024, SC_I = 8, SC_TILE = SC_T * SC_I;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* total) {
  __shared__ T ws[SC_T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T s = lane < SC_T / 32 ? ws[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const T y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const T before = (warp ? ws[warp - 1] : T(0)) + x - v;
  *total = ws[SC_T / 32 - 1];
  __syncthreads();
  return before;
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(SC_T) k_scan_tiles(const TI* __restrict__ in, long long n, TO* __restrict__ out,
                                                     TO* __restrict__ tsum) {
  const long long base = (long long)blockIdx.x * SC_TILE + (long long)threadIdx.x * SC_I;
  TO v[SC_I];
  TO s = 0;
#pragma unroll
  for (int k = 0; k < SC_I; ++k) {
    v[k] = base + k < n ? (TO)in[base + k] : TO(0);
    s += v[k];
  }
  TO total;
  TO run = block_excl_scan<TO>(s, &total);
#pragma unroll
  for (int k = 0; k < SC_I; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 0) tsum[blockIdx.x] = total;
}

template <typename TO>
__global__ void __launch_bounds__(SC_T) k_scan_sums(TO* __restrict__ tsum, long long ntiles, TO* __restrict__ grand) {
  TO carry = 0;
  for (long long c0 = 0; c0 < ntiles; c0 += SC_T) {
    const long long i = c0 + threadIdx.x;
    const TO v = i < ntiles ? tsum[i] : TO(0);
    TO total;
    const TO ex = block_excl_scan<TO>(v, &total);
    if (i < ntiles) tsum[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) *grand = carry;
}

template <typename TO>
__global__ void k_scan_add(TO* __restrict__ out, long long n, const TO* __restrict__ tsum) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] += tsum[i / SC_TILE];
}

// exclusive scan of in[0, n) into out[0, n], out[n] = total (out needs n + 1 entries)
template <typename TI, typename TO>
hp_status excl_scan(hp_ctx* ctx, const TI* in, long long n, TO* out, const char* tag) {
  const long long ntiles = std::max(1LL, (n + SC_TILE - 1) / SC_TILE);
  void* p = nullptr;
  std::string nm = std::string(tag) + ".tsum";
  HP_TRY(hp_ws(ctx, nm.c_str(), sizeof(TO) * (size_t)ntiles, &p));
  TO* tsum = (TO*)p;
  {
    ProfScope ps(ctx, "k_scan_tiles");
    k_scan_tiles<TI, TO><<<(unsigned)ntiles, SC_T, 0, ctx->stream>>>(in, n, out, tsum);
  }
  {
    ProfScope ps(ctx, "k_scan_sums");
    k_scan_sums<TO><<<1, SC_T, 0, ctx->stream>>>(tsum, ntiles, out + n);
  }
  {
    ProfScope ps(ctx, "k_scan_add");
    k_scan_add<TO><<<blocks_for(ctx, n, 256), 256, 0, ctx->stream>>>(out, n, tsum);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}

template <typename T>
hp_status read_scalar(hp_ctx* ctx, const T* dev, T* host) {
  HP_CUDA(cudaMemcpyAsync(host, dev, sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

template <typename T>
hp_status ws_arr(hp_ctx* ctx, const char* name, size_t count, T** out) {
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, name, sizeof(T) * std::max<size_t>(count, 1), &p));
  *out = (T*)p;
  return HP_OK;
}

// the CSR arrays on the device (copied when they are host memory), checked: row_ptr[0] = 0,
// non-decreasing, column indices in [0, n)
hp_status csr_view(hp_ctx* ctx, int n, const int32_t* row_ptr, const int32_t* col_idx, const double* values,
                   bool want_values, const int** rp_out, const int** ci_out, const double** val_out,
                   long long* nnz_out) {
  if (n < 1 || !row_ptr) {
    hp_set_error("sparse matrix: n >= 1 and a non-NULL row_ptr required");
    return HP_EINVAL;
  }
  const void* p = nullptr;
  HP_TRY(hp_device_view(ctx, row_ptr, sizeof(int32_t) * ((size_t)n + 1), "sp.in.rp", &p));
  const int* rp = (const int*)p;
  int ends[2] = {0, 0};
  HP_CUDA(cudaMemcpyAsync(&ends[0], rp, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaMemcpyAsync(&ends[1], rp + n, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  if (ends[0] != 0 || ends[1] < 0) {
    hp_set_error("sparse matrix: row_ptr[0] must be 0 and row_ptr[n] >= 0 (got %d, %d)", ends[0], ends[1]);
    return HP_EINVAL;
  }
  const long long nnz = ends[1];
  if (nnz && (!col_idx || (want_values && !values))) {
    hp_set_error("sparse matrix: col_idx%s NULL with %lld entries", want_values ? " or values" : "", nnz);
    return HP_EINVAL;
  }
  if (nnz) {
    HP_TRY(hp_device_view(ctx, col_idx, sizeof(int32_t) * (size_t)nnz, "sp.in.ci", &p));
  } else {   // no entries: nothing of the caller's arrays is read
    HP_TRY(hp_ws(ctx, "sp.in.none", sizeof(double), (void**)&p));
  }
  const int* ci = (const int*)p;
  if (want_values) {
    if (nnz) HP_TRY(hp_device_view(ctx, values, sizeof(double) * (size_t)nnz, "sp.in.val", &p));
    *val_out = (const double*)p;
  }
  int* bad = nullptr;
  HP_TRY(ws_arr(ctx, "sp.bad", 1, &bad));
  HP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  {
    ProfScope ps(ctx, "k_sp_validate");
    k_sp_validate<<<blocks_for(ctx, std::max<long long>(n, nnz), 256), 256, 0, ctx->stream>>>(n, rp, ci, nnz, bad);
  }
  HP_LAUNCH_CHECK();
  int b = 0;
  HP_TRY(read_scalar(ctx, bad, &b));
  if (b) {
    hp_set_error("sparse matrix: %s", (b & 1) ? "row_ptr decreases" : "a column index lies outside [0, n)");
    return HP_EINVAL;
  }
  *rp_out = rp;
  *ci_out = ci;
  *nnz_out = nnz;
  return HP_OK;
}

// ------------------------------------------------------------ Colors2Perm and colorOffsets
// Stable LSD radix sort of (key, value) pairs, 8 key bits per pass: per tile of RS_T items a
// digit histogram (digit-major over tiles), its exclusive scan, and a scatter in which an item's
// place among equal digits of its tile counts the items of earlier warps and earlier lanes.
constexpr int RS_T = 256;
static_assert(RS_T == 256, "one thread per digit in the histogram");

__global__ void __launch_bounds__(RS_T) k_rs_hist(const unsigned long long* __restrict__ key, long long n, int shift,
                                                  int ntiles, int* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long i = (long long)blockIdx.x * RS_T + threadIdx.x;
  if (i < n) atomicAdd(&h[(int)((key[i] >> shift) & 255u)], 1);
  __syncthreads();
  hist[(long long)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

__global__ void __launch_bounds__(RS_T) k_rs_scatter(const unsigned long long* __restrict__ kin,
                                                     const int* __restrict__ vin, long long n, int shift, int ntiles,
                                                     const int* __restrict__ off, unsigned long long* __restrict__ kout,
                                                     int* __restrict__ vout) {
  __shared__ int wc[RS_T / 32][256];
  for (int t = threadIdx.x; t < (RS_T / 32) * 256; t += RS_T) (&wc[0][0])[t] = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long i = (long long)blockIdx.x * RS_T + threadIdx.x;
  const bool ok = i < n;
  unsigned long long k = 0;
  int d = 0;
  if (ok) {
    k = kin[i];
    d = (int)((k >> shift) & 255u);
  }
  const unsigned int m = __match_any_sync(0xffffffffu, ok ? d : 256 + lane);   // idle lanes match nobody
  const int rank = __popc(m & ((1u << lane) - 1u));
  if (ok && rank == 0) wc[w][d] = __popc(m);
  __syncthreads();
  if (ok) {
    int before = rank;
    for (int u = 0; u < w; ++u) before += wc[u][d];
    const long long dst = (long long)off[(long long)d * ntiles + blockIdx.x] + before;
    kout[dst] = k;
    vout[dst] = vin[i];
  }
}

// sorts (key[i], val[i]), i < n, stably by the low `bits` bits of key; the result replaces the input
hp_status radix_sort_pairs(hp_ctx* ctx, unsigned long long* key, int* val, long long n, int bits, const char* tag) {
  if (n <= 1 || bits <= 0) return HP_OK;
  const long long ntiles = (n + RS_T - 1) / RS_T;
  unsigned long long* k2;
  int *v2, *hist, *off;
  const std::string t(tag);
  HP_TRY(ws_arr(ctx, (t + ".k2").c_str(), (size_t)n, &k2));
  HP_TRY(ws_arr(ctx, (t + ".v2").c_str(), (size_t)n, &v2));
  HP_TRY(ws_arr(ctx, (t + ".hist").c_str(), (size_t)(256 * ntiles), &hist));
  HP_TRY(ws_arr(ctx, (t + ".off").c_str(), (size_t)(256 * ntiles + 1), &off));
  unsigned long long *ka = key, *kb = k2;
  int *va = val, *vb = v2;
  for (int shift = 0; shift < bits; shift += 8) {
    {
      ProfScope ps(ctx, "k_rs_hist");
      k_rs_hist<<<(unsigned)ntiles, RS_T, 0, ctx->stream>>>(ka, n, shift, (int)ntiles, hist);
    }
    HP_LAUNCH_CHECK();
    HP_TRY(excl_scan(ctx, hist, 256 * ntiles, off, (t + ".scan").c_str()));
    {
      ProfScope ps(ctx, "k_rs_scatter");
      k_rs_scatter<<<(unsigned)ntiles, RS_T, 0, ctx->stream>>>(ka, va, n, shift, (int)ntiles, off, kb, vb);
    }
    HP_LAUNCH_CHECK();
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != key) {
    HP_CUDA(cudaMemcpyAsync(key, ka, sizeof(unsigned long long) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
    HP_CUDA(cudaMemcpyAsync(val, va, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  return HP_OK;
}

// The blocks of Algorithm 1 replayed from the colour paths, one level at a time: every row
// knows the first position of its block (bst, in the coordinates of the final permutation)
// and every block its size (bsz at that position).  Level 1 is the whole matrix, recorded as
// (0, n - 1, 1).
__global__ void k_ord_init(int n, int* __restrict__ bst, unsigned char* __restrict__ act, int* __restrict__ bsz,
                           int* __restrict__ ostart, int* __restrict__ oend, int* __restrict__ olev) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    bst[v] = 0;
    act[v] = 1;
    if (v == 0) {
      bsz[0] = n;
      ostart[0] = 0;
      oend[0] = n - 1;
      olev[0] = 1;
    }
  }
}

// colour count of every block of the level (colours 0 .. k - 1); a colour outside [0, block size)
// is an invalid hierarchy (flagged, not used)
__global__ void k_ord_ncol(int n, const int* __restrict__ col, const unsigned char* __restrict__ act,
                           const int* __restrict__ bst, const int* __restrict__ bsz, int* __restrict__ ncol,
                           int* __restrict__ bad) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    if (!act[v]) continue;
    const int c = col[v], b = bst[v];
    if (c < 0 || c >= bsz[b]) atomicOr(bad, 1);
    else atomicMax(ncol + b, c + 1);
  }
}

// a block recurses unless it has one colour or as many colours as rows (line 4 of the algorithm);
// the rows of each colour class of a recursing block count at slot start + colour, those of a
// stopped block at its start, so that the prefix sum keeps every block's range
__global__ void k_ord_count(int n, const int* __restrict__ col, const unsigned char* __restrict__ act,
                            const int* __restrict__ bst, const int* __restrict__ bsz, const int* __restrict__ ncol,
                            unsigned char* __restrict__ rec, int* __restrict__ cnt) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int b = bst[v];
    bool r = false;
    if (act[v]) {
      const int c = col[v], nc = ncol[b];
      r = c >= 0 && c < bsz[b] && nc != 1 && nc != bsz[b];
    }
    rec[v] = r ? 1 : 0;
    atomicAdd(cnt + b + (r ? col[v] : 0), 1);
  }
}

// the child blocks (level + 1) at their places S[slot]; the first row to reach a new block
// records (start, end, level + 1)
__global__ void k_ord_relabel(int n, int level, const int* __restrict__ col, const unsigned char* __restrict__ rec,
                              const int* __restrict__ bst, const int* __restrict__ cnt, const int* __restrict__ S,
                              int* __restrict__ nbst, int* __restrict__ nbsz, unsigned char* __restrict__ act,
                              int* __restrict__ mark, int* __restrict__ nblk, int cap, int* __restrict__ ostart,
                              int* __restrict__ oend, int* __restrict__ olev, int* __restrict__ bad) {
  const int stride = gridDim.x * blockDim.x;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const bool r = rec[v] != 0;
    const int slot = bst[v] + (r ? col[v] : 0);
    const int s = S[slot], sz = cnt[slot];
    nbst[v] = s;
    nbsz[s] = sz;
    act[v] = r ? 1 : 0;
    if (r && atomicExch(mark + s, 1) == 0) {
      const int idx = atomicAdd(nblk, 1);
      if (idx < cap) {
        ostart[idx] = s;
        oend[idx] = s + sz - 1;
        olev[idx] = level + 1;
      } else {
        atomicOr(bad, 2);
      }
    }
  }
}

__global__ void k_ord_keys(int n, const int* __restrict__ a, const int* __restrict__ lev, unsigned long long* __restrict__ key,
                           int* __restrict__ val) {
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    key[i] = lev ? (((unsigned long long)a[i] << 6) | (unsigned long long)lev[i]) : (unsigned long long)a[i];
    val[i] = i;
  }
}

__global__ void k_ord_gather(int m, const int* __restrict__ idx, const int* __restrict__ ostart,
                             const int* __restrict__ oend, const int* __restrict__ olev, int* __restrict__ out) {
  const int stride = gridDim.x * blockDim.x;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += stride) {
    const int i = idx[j];
    out[3 * (size_t)j] = ostart[i];
    out[3 * (size_t)j + 1] = oend[i];
    out[3 * (size_t)j + 2] = olev[i];
  }
}

int bits_for(long long v) {   // bits needed for values 0 .. v
  int b = 0;
  while (b < 62 && (1LL << b) <= v) ++b;
  return b;
}

}  // namespace

extern "C" hp_status hp_sparse_coloring(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                        int32_t max_levels, int32_t* paths, int32_t* radices, int32_t* n_levels) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  if (max_levels < 1 || max_levels > HP_MAX_LEVELS || !paths || !radices || !n_levels) {
    hp_set_error("hp_sparse_coloring: max_levels in [1, %d] and non-NULL outputs required", HP_MAX_LEVELS);
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  const int* rp = nullptr;
  const int* ci = nullptr;
  const double* unused = nullptr;
  long long nnz = 0;
  HP_TRY(csr_view(ctx, n, row_ptr, col_idx, nullptr, false, &rp, &ci, &unused, &nnz));

  const size_t N = (size_t)n;
  const bool paths_host = !hp_is_device_ptr(paths);
  int* P = paths;
  if (paths_host) HP_TRY(ws_arr(ctx, "sp.paths", N * max_levels, &P));
  HP_CUDA(cudaMemsetAsync(P, 0, sizeof(int) * N * max_levels, ctx->stream));

  unsigned char *act, *rec;
  int *col, *bst[2], *bsz[2], *bncol, *cnt, *S, *radix, *flag;
  unsigned int* pending;
  long long *grp[2], *hsz, *hoff, *ucnt;
  int* gci[2];
  HP_TRY(ws_arr(ctx, "sp.act", N, &act));
  HP_TRY(ws_arr(ctx, "sp.rec", N, &rec));
  HP_TRY(ws_arr(ctx, "sp.col", N, &col));
  HP_TRY(ws_arr(ctx, "sp.bst0", N, &bst[0]));
  HP_TRY(ws_arr(ctx, "sp.bst1", N, &bst[1]));
  HP_TRY(ws_arr(ctx, "sp.bsz0", N, &bsz[0]));
  HP_TRY(ws_arr(ctx, "sp.bsz1", N, &bsz[1]));
  HP_TRY(ws_arr(ctx, "sp.bncol", N, &bncol));
  HP_TRY(ws_arr(ctx, "sp.cnt", N, &cnt));
  HP_TRY(ws_arr(ctx, "sp.S", N + 1, &S));
  HP_TRY(ws_arr(ctx, "sp.radix", HP_MAX_LEVELS, &radix));
  HP_TRY(ws_arr(ctx, "sp.flag", 1, &flag));
  HP_TRY(ws_arr(ctx, "sp.pending", 1, &pending));
  HP_TRY(ws_arr(ctx, "sp.grp0", N + 1, &grp[0]));
  HP_TRY(ws_arr(ctx, "sp.grp1", N + 1, &grp[1]));
  HP_TRY(ws_arr(ctx, "sp.hsz", N, &hsz));
  HP_TRY(ws_arr(ctx, "sp.hoff", N + 1, &hoff));
  HP_TRY(ws_arr(ctx, "sp.ucnt", N, &ucnt));
  HP_TRY(ws_arr(ctx, "sp.gci0", (size_t)nnz, &gci[0]));
  HP_CUDA(cudaMemsetAsync(radix, 0, sizeof(int) * HP_MAX_LEVELS, ctx->stream));

  const int nb = blocks_for(ctx, n + 1, ST);
  {
    ProfScope ps(ctx, "k_sp_graph0");
    k_sp_graph0<<<nb, ST, 0, ctx->stream>>>(n, rp, grp[0], act, col, bst[0]);
  }
  HP_LAUNCH_CHECK();
  if (nnz) HP_CUDA(cudaMemcpyAsync(gci[0], ci, sizeof(int) * (size_t)nnz, cudaMemcpyDeviceToDevice, ctx->stream));
  HP_CUDA(cudaMemcpyAsync(bsz[0], &n, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));

  int cur = 0, levels = 0;
  for (int l = 0; l < max_levels; ++l) {
    // colour every block of level l + 1: Jones-Plassmann rounds until no active row is left
    // (each round colours at least the lowest-indexed uncoloured row, so n rounds suffice)
    const int per_check = 4;
    for (long long rounds = 0;; rounds += per_check) {
      if (rounds > (long long)n + per_check) {
        hp_set_error("hp_sparse_coloring: colouring of level %d did not finish in %lld rounds", l + 1, rounds);
        return HP_ETIMEOUT;
      }
        for (int k = 0; k < per_check; ++k) {
        if (k == per_check - 1) HP_CUDA(cudaMemsetAsync(pending, 0, sizeof(unsigned int), ctx->stream));
        ProfScope ps(ctx, "k_sp_jp");
        k_sp_jp<<<nb, ST, 0, ctx->stream>>>(n, grp[cur], gci[cur], act, col, pending);
      }
      HP_LAUNCH_CHECK();
      unsigned int left = 0;
      HP_TRY(read_scalar(ctx, pending, &left));
      if (!left) break;
    }
    HP_CUDA(cudaMemsetAsync(bncol, 0, sizeof(int) * N, ctx->stream));
    {
      ProfScope ps(ctx, "k_sp_stats");
      k_sp_stats<<<nb, ST, 0, ctx->stream>>>(n, act, col, bst[cur], bncol, radix + l, P + (size_t)l * N);
    }
    HP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * N, ctx->stream));
    HP_CUDA(cudaMemsetAsync(flag, 0, sizeof(int), ctx->stream));
    {
      ProfScope ps(ctx, "k_sp_count");
      k_sp_count<<<nb, ST, 0, ctx->stream>>>(n, act, col, bst[cur], bsz[cur], bncol, l + 1 == max_levels, rec, cnt,
                                             flag);
    }
    HP_LAUNCH_CHECK();
    levels = l + 1;
    int any = 0;
    HP_TRY(read_scalar(ctx, flag, &any));
    if (!any) break;
    // child blocks of level l + 2
    HP_TRY(excl_scan(ctx, cnt, n, S, "sp.scanS"));
    {
      ProfScope ps(ctx, "k_sp_relabel");
      k_sp_relabel<<<nb, ST, 0, ctx->stream>>>(n, rec, col, bst[cur], cnt, S, bst[cur ^ 1], bsz[cur ^ 1], act);
    }
    {
      ProfScope ps(ctx, "k_sp_hcount");
      k_sp_hcount<<<nb, ST, 0, ctx->stream>>>(n, grp[cur], gci[cur], act, bst[cur ^ 1], hsz);
    }
    HP_LAUNCH_CHECK();
    HP_TRY(excl_scan(ctx, hsz, n, hoff, "sp.scanH"));
    long long H = 0;
    HP_TRY(read_scalar(ctx, hoff + n, &H));
    int* table = nullptr;
    HP_TRY(ws_arr(ctx, "sp.table", (size_t)H, &table));
    HP_CUDA(cudaMemsetAsync(table, 0xff, sizeof(int) * (size_t)std::max(H, 1LL), ctx->stream));
    {
      ProfScope ps(ctx, "k_sp_hinsert");
      k_sp_hinsert<<<nb, ST, 0, ctx->stream>>>(n, grp[cur], gci[cur], act, bst[cur ^ 1], hoff, hsz, table, ucnt);
    }
    HP_LAUNCH_CHECK();
    HP_TRY(excl_scan(ctx, ucnt, n, grp[cur ^ 1], "sp.scanU"));
    long long E = 0;
    HP_TRY(read_scalar(ctx, grp[cur ^ 1] + n, &E));
    HP_TRY(ws_arr(ctx, cur ? "sp.gci0" : "sp.gci1", (size_t)E, &gci[cur ^ 1]));
    {
      ProfScope ps(ctx, "k_sp_hwrite");
      k_sp_hwrite<<<nb, ST, 0, ctx->stream>>>(n, hoff, hsz, table, grp[cur ^ 1], gci[cur ^ 1]);
    }
    HP_LAUNCH_CHECK();
    cur ^= 1;
  }
  std::vector<int> rad(HP_MAX_LEVELS, 0);
  HP_CUDA(cudaMemcpyAsync(rad.data(), radix, sizeof(int) * HP_MAX_LEVELS, cudaMemcpyDeviceToHost, ctx->stream));
  if (paths_host)
    HP_CUDA(cudaMemcpyAsync(paths, P, sizeof(int) * N * max_levels, cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  for (int l = 0; l < max_levels; ++l) radices[l] = l < levels ? rad[l] : 0;
  *n_levels = levels;
  return HP_OK;
}

extern "C" hp_status hp_sparse_ordering(hp_ctx* ctx, int32_t n, const int32_t* paths, int32_t n_levels,
                                        int32_t* perm, int32_t* offsets, int64_t offsets_cap, int64_t* n_offsets) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  if (n < 1 || n_levels < 0 || n_levels > HP_MAX_LEVELS || (n_levels > 0 && !paths) || (!perm && !offsets) ||
      (offsets && (offsets_cap < 0 || !n_offsets))) {
    hp_set_error("hp_sparse_ordering: n >= 1, n_levels in [0, %d], paths for n_levels > 0, an output, and "
                 "n_offsets with offsets required", HP_MAX_LEVELS);
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  const size_t N = (size_t)n;
  const int* P = nullptr;
  if (n_levels > 0) {
    const void* p = nullptr;
    HP_TRY(hp_device_view(ctx, paths, sizeof(int32_t) * N * n_levels, "ord.paths", &p));
    P = (const int*)p;
  }
  const int cap = 2 * n;   // a tree whose inner nodes have >= 2 children and <= n leaves has < 2n nodes
  unsigned char *act, *rec;
  int *bst[2], *bsz[2], *ncol, *cnt, *S, *mark, *nblk, *bad, *ostart, *oend, *olev, *val;
  unsigned long long* key;
  HP_TRY(ws_arr(ctx, "ord.act", N, &act));
  HP_TRY(ws_arr(ctx, "ord.rec", N, &rec));
  HP_TRY(ws_arr(ctx, "ord.bst0", N, &bst[0]));
  HP_TRY(ws_arr(ctx, "ord.bst1", N, &bst[1]));
  HP_TRY(ws_arr(ctx, "ord.bsz0", N, &bsz[0]));
  HP_TRY(ws_arr(ctx, "ord.bsz1", N, &bsz[1]));
  HP_TRY(ws_arr(ctx, "ord.ncol", N, &ncol));
  HP_TRY(ws_arr(ctx, "ord.cnt", N, &cnt));
  HP_TRY(ws_arr(ctx, "ord.S", N + 1, &S));
  HP_TRY(ws_arr(ctx, "ord.mark", N, &mark));
  HP_TRY(ws_arr(ctx, "ord.nblk", 1, &nblk));
  HP_TRY(ws_arr(ctx, "ord.bad", 1, &bad));
  HP_TRY(ws_arr(ctx, "ord.ostart", (size_t)cap, &ostart));
  HP_TRY(ws_arr(ctx, "ord.oend", (size_t)cap, &oend));
  HP_TRY(ws_arr(ctx, "ord.olev", (size_t)cap, &olev));
  HP_TRY(ws_arr(ctx, "ord.key", (size_t)cap, &key));
  HP_TRY(ws_arr(ctx, "ord.val", (size_t)cap, &val));
  const int one = 1;
  HP_CUDA(cudaMemcpyAsync(nblk, &one, sizeof(int), cudaMemcpyHostToDevice, ctx->stream));
  HP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
  const int nb = blocks_for(ctx, n, ST);
  k_ord_init<<<nb, ST, 0, ctx->stream>>>(n, bst[0], act, bsz[0], ostart, oend, olev);
  HP_LAUNCH_CHECK();
  int cur = 0;
  for (int l = 0; l < n_levels; ++l) {
    const int* col = P + (size_t)l * N;
    HP_CUDA(cudaMemsetAsync(ncol, 0, sizeof(int) * N, ctx->stream));
    HP_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * N, ctx->stream));
    HP_CUDA(cudaMemsetAsync(mark, 0, sizeof(int) * N, ctx->stream));
    {
      ProfScope ps(ctx, "k_ord_level");
      k_ord_ncol<<<nb, ST, 0, ctx->stream>>>(n, col, act, bst[cur], bsz[cur], ncol, bad);
      k_ord_count<<<nb, ST, 0, ctx->stream>>>(n, col, act, bst[cur], bsz[cur], ncol, rec, cnt);
    }
    HP_LAUNCH_CHECK();
    HP_TRY(excl_scan(ctx, cnt, n, S, "ord.scan"));
    {
      ProfScope ps(ctx, "k_ord_level");
      k_ord_relabel<<<nb, ST, 0, ctx->stream>>>(n, l + 1, col, rec, bst[cur], cnt, S, bst[cur ^ 1], bsz[cur ^ 1], act,
                                                mark, nblk, cap, ostart, oend, olev, bad);
    }
    HP_LAUNCH_CHECK();
    cur ^= 1;
  }
  int flags = 0, m = 0;
  HP_TRY(read_scalar(ctx, bad, &flags));
  HP_TRY(read_scalar(ctx, nblk, &m));
  if (flags) {
    hp_set_error("hp_sparse_ordering: %s", (flags & 1) ? "a colour lies outside [0, size of its block)"
                                                       : "more blocks than a hierarchy of n rows has");
    return HP_EINVAL;
  }
  if (perm) {   // rows by the first position of their last block, ties (rows of one block) by index
    k_ord_keys<<<nb, ST, 0, ctx->stream>>>(n, bst[cur], nullptr, key, val);
    HP_LAUNCH_CHECK();
    HP_TRY(radix_sort_pairs(ctx, key, val, n, bits_for(n), "ord.rs"));
    HP_CUDA(cudaMemcpyAsync(perm, val, sizeof(int) * N, cudaMemcpyDefault, ctx->stream));
  }
  if (offsets) {   // pre-order of the recursion: by start, a block before its first child (level)
    *n_offsets = m;
    if (m > offsets_cap) {
      HP_CUDA(cudaStreamSynchronize(ctx->stream));
      hp_set_error("hp_sparse_ordering: %d blocks, offsets_cap %lld (2n - 1 always suffices)", m,
                   (long long)offsets_cap);
      return HP_EINVAL;
    }
    k_ord_keys<<<blocks_for(ctx, m, ST), ST, 0, ctx->stream>>>(m, ostart, olev, key, val);
    HP_LAUNCH_CHECK();
    HP_TRY(radix_sort_pairs(ctx, key, val, m, bits_for(n) + 6, "ord.rs"));
    int* out = offsets;
    const bool host = !hp_is_device_ptr(offsets);
    if (host) HP_TRY(ws_arr(ctx, "ord.out", 3 * (size_t)m, &out));
    k_ord_gather<<<blocks_for(ctx, m, ST), ST, 0, ctx->stream>>>(m, val, ostart, oend, olev, out);
    HP_LAUNCH_CHECK();
    if (host) HP_CUDA(cudaMemcpyAsync(offsets, out, sizeof(int) * 3 * (size_t)m, cudaMemcpyDeviceToHost, ctx->stream));
  } else if (n_offsets) {
    *n_offsets = m;
  }
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

namespace {

__global__ void k_sp_check_paths(LatGeom g, long long total, int* __restrict__ bad) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
    const int c = g.paths[i];
    if (c < 0 || c >= g.radix[i / g.V]) atomicOr(bad, 1);
  }
}

__global__ void k_sp_phases(LatGeom g, uint32_t first, int count, uint16_t* __restrict__ out) {
  const long long total = (long long)count * g.V;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    const int j = (int)(t / g.V);
    const uint32_t i = (uint32_t)(t - (long long)j * g.V);
    out[t] = (uint16_t)probe_phase(g, i, first + (uint32_t)j);
  }
}

}  // namespace

// Geometry of a general sparse matrix for the probing kernels and the CG engine.  The
// hierarchical sequence (probe_kind 0) uses the levels that the vectors m < s_end resolve,
// k = min{k : c(1) ... c(k) >= s_end}, with period P = lcm(2, c(1), ..., c(k)); the natural
// and Z_2 sequences use P = 2.  The paths of those levels are checked against the radices.
hp_status hp_sparse_geom(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* values,
                         const int32_t* paths, const int32_t* radices, int32_t n_levels, int64_t s_end,
                         int32_t probe_kind, LatGeom* g) {
  memset(g, 0, sizeof(*g));
  if (n < 1) {
    hp_set_error("sparse matrix: n must be >= 1");
    return HP_EINVAL;
  }
  g->V = n;
  g->nd = 1;
  g->L[0] = n;
  for (int j = 1; j < 8; ++j) g->L[j] = 1;
  g->op_kind = HP_OP_LAPLACIAN;
  g->dof = 1;
  g->probe_kind = probe_kind;
  if (row_ptr) {
    const int* rp = nullptr;
    const int* ci = nullptr;
    const double* val = nullptr;
    long long nnz = 0;
    HP_TRY(csr_view(ctx, n, row_ptr, col_idx, values, true, &rp, &ci, &val, &nnz));
    g->csr_rp = rp;
    g->csr_ci = ci;
    g->csr_val = val;
  }
  long long P = 2;
  if (probe_kind == HP_PROBE_HIERARCHICAL) {
    if (n_levels < 0 || n_levels > HP_MAX_LEVELS || (n_levels > 0 && (!paths || !radices))) {
      hp_set_error("colour hierarchy: n_levels in [0, %d] with non-NULL paths and radices required", HP_MAX_LEVELS);
      return HP_EINVAL;
    }
    long long gamma = 1;
    int k = 0;
    while (gamma < s_end && k < n_levels) {
      if (radices[k] < 1 || radices[k] > n) {
        hp_set_error("colour hierarchy: radix of level %d is %d", k + 1, radices[k]);
        return HP_EINVAL;
      }
      gamma *= radices[k];
      ++k;
    }
    if (gamma < s_end) {
      hp_set_error("the hierarchy resolves %lld probing vectors, fewer than the %lld asked for", gamma,
                   (long long)s_end);
      return HP_EUNSUPPORTED;
    }
    for (int l = 0; l < k; ++l) {
      P = std::lcm(P, (long long)radices[l]);
      if (P > 65535) {
        hp_set_error("the period lcm(2, c(1..%d)) exceeds 65535", l + 1);
        return HP_EUNSUPPORTED;
      }
    }
    g->nlev = k;
    const void* p = nullptr;
    HP_TRY(hp_ws(ctx, "sp.radix", sizeof(int) * HP_MAX_LEVELS, (void**)&p));
    if (k) HP_CUDA(cudaMemcpyAsync((void*)p, radices, sizeof(int) * k, cudaMemcpyHostToDevice, ctx->stream));
    g->radix = (const int*)p;
    if (k) {
      HP_TRY(hp_device_view(ctx, paths, sizeof(int32_t) * (size_t)n * k, "sp.in.paths", &p));
    } else {   // one vector (z_0 itself): the digit loop reads no path, but the pointer marks the kind
      HP_TRY(hp_ws(ctx, "sp.nopath", sizeof(int), (void**)&p));
    }
    g->paths = (const int*)p;
    if (k) {
      int* bad = nullptr;
      HP_TRY(ws_arr(ctx, "sp.bad", 1, &bad));
      HP_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), ctx->stream));
      const long long total = (long long)n * k;
      {
        ProfScope ps(ctx, "k_sp_check_paths");
        k_sp_check_paths<<<blocks_for(ctx, total, 256), 256, 0, ctx->stream>>>(*g, total, bad);
      }
      HP_LAUNCH_CHECK();
      int b = 0;
      HP_TRY(read_scalar(ctx, bad, &b));
      if (b) {
        hp_set_error("colour hierarchy: a colour lies outside [0, c(l))");
        return HP_EINVAL;
      }
    }
  } else if (probe_kind == HP_PROBE_NATURAL) {
    if (n & (n - 1)) {
      hp_set_error("Hadamard vectors in natural order need n a power of two (n = %d)", n);
      return HP_EUNSUPPORTED;
    }
    g->K = 31 - __builtin_clz((unsigned)n);
  } else if (probe_kind != HP_PROBE_Z2) {
    hp_set_error("unknown probe kind %d", probe_kind);
    return HP_EINVAL;
  }
  g->P = (int)P;
  g->parts = P > 2 ? 2 : 1;
  std::vector<double> tab(2 * (size_t)P);
  HP_TRY(hp_phase_values((int32_t)P, tab.data()));
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "sp.ptab", sizeof(double2) * (size_t)P, &p));
  HP_CUDA(cudaMemcpyAsync(p, tab.data(), sizeof(double2) * (size_t)P, cudaMemcpyHostToDevice, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));   // the host table must outlive the copy
  g->ptab = (const double2*)p;
  return HP_OK;
}

extern "C" hp_status hp_sparse_probe_vectors(hp_ctx* ctx, int32_t n, const int32_t* paths, const int32_t* radices,
                                             int32_t n_levels, int64_t first, int64_t count, uint64_t z0_seed,
                                             uint16_t* phase_dev, int32_t* period_out) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  if (first < 0 || count < 0 || first + count > (int64_t)n) {
    hp_set_error("probe range [%lld, %lld) outside [0, n = %d]", (long long)first, (long long)(first + count), n);
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  LatGeom g;
  HP_TRY(hp_sparse_geom(ctx, n, nullptr, nullptr, nullptr, paths, radices, n_levels, std::max<int64_t>(first + count, 1),
                        HP_PROBE_HIERARCHICAL, &g));
  g.z0_seed = z0_seed;
  if (period_out) *period_out = g.P;
  if (count == 0) return HP_OK;
  if (!phase_dev || !hp_is_device_ptr(phase_dev)) {
    hp_set_error("hp_sparse_probe_vectors: phase_dev must be device memory");
    return HP_EINVAL;
  }
  {
    ProfScope ps(ctx, "k_sp_phases");
    k_sp_phases<<<blocks_for(ctx, count * (long long)n, 256), 256, 0, ctx->stream>>>(g, (uint32_t)first, (int)count,
                                                                                     phase_dev);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}
