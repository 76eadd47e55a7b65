// Internal declarations of the hierarchical-probing library (not installed).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <map>
#include <memory>
#include <string>
#include <vector>

#include "../../include/hprobe.h"

// ------------------------------------------------------------------ errors
void hp_set_error(const char* fmt, ...);

#define HP_CUDA(call)                                                                       \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      hp_set_error("%s failed at %s:%d: %s", #call, __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return HP_ECUDA;                                                                      \
    }                                                                                       \
  } while (0)

#define HP_TRY(expr)                     \
  do {                                   \
    hp_status s_ = (expr);               \
    if (s_ != HP_OK) return s_;          \
  } while (0)

#define HP_LAUNCH_CHECK()                                                                   \
  do {                                                                                      \
    cudaError_t e_ = cudaGetLastError();                                                    \
    if (e_ != cudaSuccess) {                                                                \
      hp_set_error("kernel launch failed at %s:%d: %s", __FILE__, __LINE__, cudaGetErrorString(e_)); \
      return HP_ECUDA;                                                                      \
    }                                                                                       \
  } while (0)

// -------------------------------------------------------------- precisions
// PRFF: float-float (an unevaluated sum hi + lo of two FP32 numbers, 48-bit significand)
enum { PR64 = 0, PR32 = 1, PR16 = 2, PRB16 = 3, PRFF = 4 };

// ---------------------------------------------------------- lattice (device)
// Everything a kernel needs about one lattice: geometry, probing basis and
// operator.  Plain data, copied to device memory as an array (one entry per
// lattice of a batch).
#define HP_MAX_LEVELS 32   // levels of a colour hierarchy of a general sparse matrix

struct LatGeom {
  int nd;                 // number of dimensions (operators: padded to 4)
  int L[8];
  int V;
  int ks[8];              // 2-adic valuation of each size
  int kmax, K;            // binary levels
  int Q, R, P;            // odd block size, final level size (0: unequal), period
  int qstride[8];         // strides of the q-torus (sizes p_j)
  unsigned long long z0_seed;
  int probe_kind;         // hp_probe_kind: hierarchical (0), natural-order Hadamard (1), Z_2 noise (2)
  // a general sparse matrix (Algorithm 1 path): CSR rows of A, and the colour hierarchy that
  // defines the probing vectors (paths[l * V + i] = colour of row i at level l + 1)
  const int* csr_rp;
  const int* csr_ci;
  const double* csr_val;
  const int* paths;
  int nlev;
  const int* radix;       // [nlev] colour counts c(l) in device memory (an array here would be
                          // indexed dynamically and move the whole struct to local memory)
  // deflation (Laplacian): k orthonormal eigenvectors [k][V] in device memory; sources are
  // projected, b -> b - V (V^T b)
  const double* defl_V;
  int defl_k;
  double quad_tol;        // Laplacian CG: > 0 stops on the quadrature bracket (Gauss / Gauss-Radau)
  double quad_mu;         // the Gauss-Radau node, 0 < quad_mu <= lambda_min(A)
  const uint32_t* loc;    // [V] hierarchical position of each site
  const int32_t* wtab;    // [Q] position inside the odd block of each q point
  const double2* ptab;    // [P] (cos, sin) of 2 pi k / P
  // operator
  int op_kind;
  double kappa, mass;
  const double* mass_field;   // [V] or nullptr
  const float* mass_field32;  // FP32 copy of mass_field for the FP32-arithmetic kernels
  float diag0;                // 1 + mass in FP32
  const double2* U64;         // [4][9][V]
  const float4* U32;          // [4][3][V]  first two rows
  const uint2* U16;           // [4][3][V]  first two rows, binary16
  const float4* U32f;         // [4][4][V]  entries 0-7 of the full link, FP32
  const float2* U32g;         // [4][V]     entry 8
  const uint4* U16f;          // [4][2][V]  entries 0-7 of the full link, binary16
  const unsigned int* U16g;   // [4][V]     entry 8
  const float4* U32fl;        // [4][4][V]  low parts (u - (float)u) of entries 0-7, float-float links
  const float2* U32gl;        // [4][V]     low part of entry 8
  // clover term: A(x) = (1 + m + mu(x)) + C(x) (Wilson diagonal plus the Sheikholeslami-Wohlert
  // term) as two Hermitian 6x6 blocks per site (spins 0-1 and 2-3: C commutes with gamma_5),
  // each packed as 6 real diagonal entries then the 15 entries above the diagonal (row-major)
  // as (re, im): 36 reals per block, 72 per site; Ai* hold A(x)^-1 in the same form.
  int clover;                 // 1: the diagonal is A(x) (arrays below), 0: 1 + m + mu(x)
  const double2* A64;         // [36][V]
  const float4* A32;          // [18][V]
  const float4* A32l;         // [18][V] low parts (float-float)
  const double2* Ai64;
  const float4* Ai32;
  const float4* Ai32l;
  int dof;                    // unknowns per site that carry a source (12 Wilson, 1 Laplacian)
  int parts;                  // Laplacian: 2 when probes are complex (re, im solved apart)
};

// ------------------------------------------------------------- slot state
enum { SLOT_EMPTY = 0, SLOT_INIT = 1, SLOT_RUN = 2, SLOT_DONE = 3, SLOT_FAIL = 4 };

struct SlotState {
  double2 alpha, beta, omega, rho;   // BiCGStab scalars (CG uses .x)
  double bnorm2, rnorm2, rmax2, true_res2;
  double rexact2;                    // ||r||^2 at the last FP64 true residual
  double gauss, radau;               // CG quadrature bounds: Gauss sum G_k, Gauss-Radau coefficient
  double pad_d;
  double2 q;                         // quadrature v^H x at harvest
  int status, need_update, restart, iters;   // need_update: 1 group (FP32) update, 2 FP64 true residual
  int updates, lat, a, m;            // lattice index, dilution index / part, probe index
  int sloppy_mv, fp64_mv, gupdates, pad1;
};

// ------------------------------------------------------------- the context
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

struct LatticeSetup {
  std::vector<int64_t> dims;
  LatGeom g;                // device pointers filled
  DevBuf loc, wtab, ptab;
  int64_t n_vectors = 0;
  bool equal = false;
};

struct ProfRecord {
  std::string name;
  cudaEvent_t a, b;
};

struct hp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  std::map<std::vector<int64_t>, std::unique_ptr<LatticeSetup>> lattices;
  std::map<std::string, DevBuf> ws;          // named grow-only workspace
  bool profiling = false;
  std::vector<ProfRecord> prof;
  std::vector<cudaEvent_t> event_pool;
  std::map<std::string, int> autotune;       // key -> threads per block
  long long launches = 0;                    // kernels launched (graph replays included)
  // clover blocks kept per workspace tag: rebuilt only when the links, mass field or
  // coefficients they came from change (a 64-bit hash of the input bits is compared)
  struct CloverKey {
    unsigned long long hash = 0;
    double csw = 0, kappa = 0, mass = 0;
    int V = 0;
    const void* buf = nullptr;
  };
  std::map<std::string, CloverKey> clover_keys;
};

// workspace
hp_status hp_ws(hp_ctx* ctx, const char* name, size_t bytes, void** out);
hp_status hp_ws_free_all(hp_ctx* ctx);

// profiling around a launch
void hp_prof_begin(hp_ctx* ctx, const char* name, cudaEvent_t* a);
void hp_prof_end(hp_ctx* ctx, const char* name, cudaEvent_t a);
struct ProfScope {
  hp_ctx* ctx;
  const char* name;
  cudaEvent_t a = nullptr;
  ProfScope(hp_ctx* c, const char* n) : ctx(c), name(n) {
    ctx->launches += 1;
    hp_prof_begin(ctx, name, &a);
  }
  ~ProfScope() { hp_prof_end(ctx, name, a); }
};

// grid-stride launches: enough blocks for n items, at most 16 per SM
static inline int blocks_for(hp_ctx* ctx, long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)ctx->num_sms * 16;
  return (int)std::max(1LL, std::min(b, cap));
}

// general sparse matrix (hp_sparse.cu): geometry of the CSR operator and its probing sequence
// for vectors m < s_end (row_ptr may be NULL for the probing vectors alone)
hp_status hp_sparse_geom(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx, const double* values,
                         const int32_t* paths, const int32_t* radices, int32_t n_levels, int64_t s_end,
                         int32_t probe_kind, LatGeom* g);

// lattice setup (hp_core.cu)
hp_status hp_validate_lattice(const hp_lattice* lat, int max_nd, std::vector<int64_t>* dims);
hp_status hp_get_lattice(hp_ctx* ctx, const std::vector<int64_t>& dims, LatticeSetup** out);

// host/device buffers: returns a device pointer to the data (copying host data
// into workspace `name` when needed)
hp_status hp_device_view(hp_ctx* ctx, const void* p, size_t bytes, const char* name, const void** out);
// A view of p for ONE streaming read by a kernel: device memory as is; pinned host memory that is
// mapped into the device address space (cudaHostAlloc, cudaHostRegister) is read in place over the
// host link, with no staging copy; other host memory is copied like hp_device_view.
hp_status hp_stream_view(hp_ctx* ctx, const void* p, size_t bytes, const char* name, const void** out);
bool hp_is_device_ptr(const void* p);

// operator preparation (hp_wilson.cu): converts links to the internal
// layouts of `geom` (allocated in workspace under `tag`)
hp_status hp_prepare_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom* geom, const char* tag, int need_prec);
hp_status hp_prepare_mass(hp_ctx* ctx, const hp_operator* op, LatGeom* geom, const char* tag);
// clover blocks A and A^-1 (hp_clover.cu); needs the FP64 links U64 and the mass field of `geom`
hp_status hp_prepare_clover(hp_ctx* ctx, const hp_operator* op, LatGeom* geom, const char* tag);

// ------------------------------------------------------------- solver API
struct SolveProblem {
  std::vector<LatGeom> lats;       // device pointers set
  std::vector<int64_t> s_max;      // probes per lattice
  std::vector<int64_t> first;      // first probe per lattice
  double tol;
  hp_solver_opts opts;
  bool want_grad = false;
  std::vector<double*> grad_dev;   // per lattice, [V] accumulators (device)
  double2* x_keep = nullptr;       // optional: solutions of the first n_keep right-hand sides of lattice 0
  int64_t n_keep = 0;              // (device, complex [n_keep][V][12], right-hand side (m - first) dof + a)
};

struct SolveResult {
  std::vector<std::vector<double2>> qj;   // per lattice, per right-hand side (m*dof+a)
  std::vector<std::vector<double2>> qb;   // CG quadrature bounds (lower, upper) in the same order
  hp_solve_stats stats;
  bool unconverged = false;
};

// implemented per operator family
hp_status hp_solve_wilson(hp_ctx* ctx, SolveProblem& pb, SolveResult& res);
hp_status hp_solve_laplace(hp_ctx* ctx, SolveProblem& pb, SolveResult& res);

// -------------------------------------------------------- device helpers
#ifdef __CUDACC__

__device__ __forceinline__ unsigned long long splitmix64_at(unsigned long long seed, unsigned long long index) {
  unsigned long long z = seed + (index + 1ull) * 0x9E3779B97F4A7C15ull;   // output number `index`
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ int probe_phase(const LatGeom& g, uint32_t site, uint32_t m) {
  if (g.paths) {   // general sparse matrix: mixed-radix digits of m against the colour path of the row
    int ph = 0;
    uint32_t rest = m;
    for (int l = 0; l < g.nlev; ++l) {
      const uint32_t r = (uint32_t)g.radix[l];
      const uint32_t d = rest % r;
      rest /= r;
      ph += (g.P / (int)r) * (int)((d * (uint32_t)g.paths[(size_t)l * g.V + site]) % r);
    }
    if (g.z0_seed && (splitmix64_at(g.z0_seed, site) >> 63)) ph += g.P >> 1;
    return ph % g.P;
  }
  if (g.probe_kind == HP_PROBE_Z2)   // independent Z_2 noise: top bit of output m V + site
    return (splitmix64_at(g.z0_seed, (unsigned long long)m * (unsigned long long)g.V + site) >> 63) ? (g.P >> 1) : 0;
  if (g.probe_kind == HP_PROBE_NATURAL) {   // Sylvester Hadamard H(site, m), natural order (V = 2^K)
    int ph = (__popc(site & m) & 1) * (g.P >> 1);
    if (g.z0_seed && (splitmix64_at(g.z0_seed, site) >> 63)) ph += g.P >> 1;
    return ph % g.P;
  }
  uint32_t loc = g.loc[site];
  uint32_t lb = loc, w = 0;
  if (g.Q > 1) {
    lb = loc / (uint32_t)g.Q;
    w = loc - lb * (uint32_t)g.Q;
  }
  int ph = 0;
  uint32_t hi = m;
  if (g.K > 0) {
    uint32_t ebin = m & ((1u << g.K) - 1u);
    hi = m >> g.K;
    uint32_t col = __brev(ebin) >> (32 - g.K);       // Hperm(m) = bit reversal over K bits
    ph = (__popc(lb & col) & 1) * (g.P >> 1);
  }
  if (hi > 0 && g.R > 0) {                             // three-colour level and final Fourier level
    uint32_t e3 = hi % 3u, ef = hi / 3u;
    uint32_t C = w / (uint32_t)g.R, r = w - C * (uint32_t)g.R;
    ph += (g.P / 3) * (int)((C * e3) % 3u);
    ph += (g.P / g.R) * (int)((unsigned long long)r * ef % (unsigned long long)g.R);
  }
  if (g.z0_seed && (splitmix64_at(g.z0_seed, site) >> 63)) ph += g.P >> 1;
  return ph % g.P;
}

template <typename T>
struct cplx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cplx<T> cconjmul(cplx<T> a, cplx<T> b) {  // conj(a) * b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}

// block-level deterministic reduction helpers (fixed shuffle tree, fixed warp order)
template <int NQ, int NTHREADS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NQ], double* out_q0, size_t q_stride) {
  __shared__ double sh[NQ][NTHREADS / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double t = v[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[q][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double t = 0.0;
      for (int w = 0; w < NTHREADS / 32; ++w) t += sh[q][w];
      out_q0[q * q_stride] = t;
    }
  }
}

// returns true in every thread of the block that finishes last for this slot
__device__ __forceinline__ bool last_block(unsigned int* counter, unsigned int nparts) {
  __shared__ int am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int t = atomicAdd(counter, 1u);
    am_last = (t == nparts - 1u);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last != 0;
}

// sum of partials[q][0..nparts) in a fixed order by one block; result in every thread's out[q]
template <int NQ, int NTHREADS>
__device__ __forceinline__ void block_sum_partials(const double* part, size_t q_stride, int nparts, double (&out)[NQ]) {
  __shared__ double sh2[NQ][NTHREADS];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    double t = 0.0;
    for (int i = threadIdx.x; i < nparts; i += NTHREADS) t += __ldcg(part + q * q_stride + i);
    sh2[q][threadIdx.x] = t;
  }
  __syncthreads();
  for (int s = NTHREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
#pragma unroll
      for (int q = 0; q < NQ; ++q) sh2[q][threadIdx.x] += sh2[q][threadIdx.x + s];
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < NQ; ++q) out[q] = sh2[q][0];
  __syncthreads();
}

#endif  // __CUDACC__
