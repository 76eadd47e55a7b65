// Context, errors, workspace, profiling, lattice set-up, and the two
// integer kernels of the method: the hierarchical permutation (Section 3,
// Algorithm 5 in closed form; Section 3.4 for odd factors) and the probing
// vectors (Section 2.2, Eqs. HpermSequence / row-col-permutation /
// Hperm-general-recursive; Section 4, Eq. removebias).
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <cmath>

#include "hp_internal.h"

// ------------------------------------------------------------------ errors
static thread_local char g_err[1024] = "no error";

void hp_set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

extern "C" const char* hp_last_error(void) { return g_err; }

// ------------------------------------------------------------------ context
extern "C" hp_status hp_ctx_create(int device, void* cuda_stream, hp_ctx** out) {
  if (!out) {
    hp_set_error("hp_ctx_create: out is NULL");
    return HP_EINVAL;
  }
  *out = nullptr;
  int n = 0;
  HP_CUDA(cudaGetDeviceCount(&n));
  if (device < 0 || device >= n) {
    hp_set_error("hp_ctx_create: device %d not in [0, %d)", device, n);
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(device));
  hp_ctx* c = new hp_ctx();
  c->device = device;
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) {
    delete c;
    hp_set_error("cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    return HP_ECUDA;
  }
  c->num_sms = prop.multiProcessorCount;
  if (cuda_stream) {
    c->stream = (cudaStream_t)cuda_stream;
  } else {
    // a blocking stream: ordered with work on the legacy default stream of the caller
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamDefault);
    if (e != cudaSuccess) {
      delete c;
      hp_set_error("cudaStreamCreate: %s", cudaGetErrorString(e));
      return HP_ECUDA;
    }
    c->own_stream = true;
  }
  *out = c;
  return HP_OK;
}

extern "C" void hp_ctx_destroy(hp_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->lattices) {
    cudaFree(kv.second->loc.p);
    cudaFree(kv.second->wtab.p);
    cudaFree(kv.second->ptab.p);
  }
  hp_ws_free_all(ctx);
  for (auto& r : ctx->prof) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto ev : ctx->event_pool) cudaEventDestroy(ev);
  if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

extern "C" hp_status hp_ctx_synchronize(hp_ctx* ctx) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

hp_status hp_ws(hp_ctx* ctx, const char* name, size_t bytes, void** out) {
  DevBuf& b = ctx->ws[name];
  if (b.bytes < bytes) {
    if (b.p) {
      HP_CUDA(cudaStreamSynchronize(ctx->stream));
      HP_CUDA(cudaFree(b.p));
      b.p = nullptr;
      b.bytes = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      hp_set_error("workspace '%s': cudaMalloc of %zu bytes failed: %s", name, bytes, cudaGetErrorString(e));
      b.p = nullptr;
      return HP_ENOMEM;
    }
    b.bytes = bytes;
  }
  *out = b.p;
  return HP_OK;
}

hp_status hp_ws_free_all(hp_ctx* ctx) {
  for (auto& kv : ctx->ws)
    if (kv.second.p) cudaFree(kv.second.p);
  ctx->ws.clear();
  return HP_OK;
}

bool hp_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

hp_status hp_device_view(hp_ctx* ctx, const void* p, size_t bytes, const char* name, const void** out) {
  if (hp_is_device_ptr(p)) {
    *out = p;
    return HP_OK;
  }
  void* d = nullptr;
  HP_TRY(hp_ws(ctx, name, bytes, &d));
  HP_CUDA(cudaMemcpyAsync(d, p, bytes, cudaMemcpyHostToDevice, ctx->stream));
  *out = d;
  return HP_OK;
}

hp_status hp_stream_view(hp_ctx* ctx, const void* p, size_t bytes, const char* name, const void** out) {
  cudaPointerAttributes a;
  if (p && cudaPointerGetAttributes(&a, p) == cudaSuccess && a.type == cudaMemoryTypeHost && a.devicePointer) {
    *out = a.devicePointer;   // pinned host memory mapped into the device: read in place
    return HP_OK;
  }
  cudaGetLastError();
  return hp_device_view(ctx, p, bytes, name, out);
}

// ---------------------------------------------------------------- profiling
static cudaEvent_t take_event(hp_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

void hp_prof_begin(hp_ctx* ctx, const char* name, cudaEvent_t* a) {
  (void)name;
  if (!ctx->profiling) return;
  *a = take_event(ctx);
  cudaEventRecord(*a, ctx->stream);
}

void hp_prof_end(hp_ctx* ctx, const char* name, cudaEvent_t a) {
  if (!ctx->profiling || !a) return;
  cudaEvent_t b = take_event(ctx);
  cudaEventRecord(b, ctx->stream);
  ctx->prof.push_back({name, a, b});
}

extern "C" hp_status hp_profile_enable(hp_ctx* ctx, int32_t on) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  ctx->profiling = on != 0;
  return HP_OK;
}

extern "C" hp_status hp_launch_count(hp_ctx* ctx, int64_t* out) {
  if (!ctx || !out) {
    hp_set_error("hp_launch_count: NULL argument");
    return HP_EINVAL;
  }
  *out = ctx->launches;
  return HP_OK;
}

extern "C" hp_status hp_profile_report(hp_ctx* ctx, char* buf, int64_t size) {
  if (!ctx || !buf || size < 3) {
    hp_set_error("hp_profile_report: bad arguments");
    return HP_EINVAL;
  }
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  std::map<std::string, std::pair<long, double>> agg;
  for (auto& r : ctx->prof) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    auto& e = agg[r.name];
    e.first += 1;
    e.second += ms;
    ctx->event_pool.push_back(r.a);
    ctx->event_pool.push_back(r.b);
  }
  ctx->prof.clear();
  std::string s = "{";
  bool firstk = true;
  for (auto& kv : agg) {
    char line[256];
    snprintf(line, sizeof(line), "%s\"%s\": {\"launches\": %ld, \"ms\": %.6f}", firstk ? "" : ", ", kv.first.c_str(),
             kv.second.first, kv.second.second);
    s += line;
    firstk = false;
  }
  // autotuner decisions (stencil right-hand sides per thread, per lattice/precision/slot count)
  s += firstk ? "\"_autotune\": {" : ", \"_autotune\": {";
  bool firsta = true;
  for (auto& kv : ctx->autotune) {
    char line[256];
    snprintf(line, sizeof(line), "%s\"%s\": %d", firsta ? "" : ", ", kv.first.c_str(), kv.second);
    s += line;
    firsta = false;
  }
  s += "}}";
  size_t n = s.size() < (size_t)(size - 1) ? s.size() : (size_t)(size - 1);
  memcpy(buf, s.data(), n);
  buf[n] = 0;
  return HP_OK;
}

// ------------------------------------------------------- lattice set-up (host)
hp_status hp_validate_lattice(const hp_lattice* lat, int max_nd, std::vector<int64_t>* dims) {
  if (!lat) {
    hp_set_error("lattice is NULL");
    return HP_EINVAL;
  }
  if (lat->ndim < 1 || lat->ndim > max_nd) {
    hp_set_error("ndim = %d outside [1, %d]", lat->ndim, max_nd);
    return HP_EINVAL;
  }
  int64_t V = 1;
  dims->clear();
  for (int j = 0; j < lat->ndim; ++j) {
    if (lat->dims[j] < 1) {
      hp_set_error("dims[%d] = %lld < 1", j, (long long)lat->dims[j]);
      return HP_EINVAL;
    }
    V *= lat->dims[j];
    if (V > (int64_t(1) << 31)) {
      hp_set_error("lattice volume exceeds 2^31");
      return HP_EINVAL;
    }
    dims->push_back(lat->dims[j]);
  }
  return HP_OK;
}

// Colour of the three-colouring theorem (Section 3.4) on the q-torus.
static int three_colour(const int* q, const int* n, int nd) {
  int s = 0;
  for (int j = 0; j < nd; ++j) s += q[j] + ((q[j] == n[j] - 1 && (n[j] - 1) % 3 == 0) ? 1 : 0);
  return s % 3;
}

// --- double-double arithmetic for the (cos, sin) table (error-free transformations)
struct dd {
  double hi, lo;
};
static dd two_sum(double a, double b) {
  double s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}
static dd dd_add(dd a, dd b) {
  dd s = two_sum(a.hi, b.hi);
  double lo = s.lo + a.lo + b.lo;
  return two_sum(s.hi, lo);
}
static dd dd_mul(dd a, dd b) {
  double p = a.hi * b.hi;
  double e = std::fma(a.hi, b.hi, -p);
  e += a.hi * b.lo + a.lo * b.hi;
  return two_sum(p, e);
}
static dd dd_mul_d(dd a, double b) { return dd_mul(a, dd{b, 0.0}); }
static dd dd_div_d(dd a, double b) {
  double q1 = a.hi / b;
  dd r = dd_add(a, dd_mul_d(dd{q1, 0.0}, -b));
  double q2 = r.hi / b;
  return two_sum(q1, q2);
}
// cos and sin of x in [0, pi/4] by their Taylor series in double-double
static void dd_cos_sin(dd x, double* c, double* s) {
  dd x2 = dd_mul(x, x);
  dd cs = {1.0, 0.0}, sn = x;
  dd tc = {1.0, 0.0}, ts = x;
  for (int k = 1; k < 30; ++k) {
    tc = dd_div_d(dd_mul(tc, x2), -(double)((2 * k - 1) * (2 * k)));
    ts = dd_div_d(dd_mul(ts, x2), -(double)((2 * k) * (2 * k + 1)));
    cs = dd_add(cs, tc);
    sn = dd_add(sn, ts);
    if (std::fabs(tc.hi) < 1e-40 && std::fabs(ts.hi) < 1e-40) break;
  }
  *c = cs.hi;
  *s = sn.hi;
}

// cos, sin of 2 pi k / P: exact octant reduction in integers, then a
// double-double series, then one rounding to binary64.
static void phase_value(int k, int P, double* cv, double* sv) {
  const dd PI = {3.141592653589793116, 1.2246467991473532072e-16};
  long long e8 = 8LL * k;
  int o = (int)(e8 / P);
  long long f = e8 % P;   // angle = (pi/4) (o + f/P)
  bool odd = o & 1;
  long long num = odd ? (P - f) : f;   // reduced angle phi = (pi/4) num / P
  double c = 1.0, s = 0.0;
  if (num != 0) {
    dd phi = dd_div_d(dd_mul_d(PI, (double)num), 4.0 * (double)P);
    dd_cos_sin(phi, &c, &s);
  }
  double C, S;
  switch (o) {
    case 0: C = c; S = s; break;
    case 1: C = s; S = c; break;
    case 2: C = -s; S = c; break;
    case 3: C = -c; S = s; break;
    case 4: C = -c; S = -s; break;
    case 5: C = -s; S = -c; break;
    case 6: C = s; S = -c; break;
    default: C = c; S = -s; break;
  }
  *cv = C + 0.0;   // no negative zero
  *sv = S + 0.0;
}

static int64_t gcd64(int64_t a, int64_t b) {
  while (b) {
    int64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}

struct BasisFacts {
  int nd, V, K, kmax, Q, R, P;
  int L[8], ks[8], ps[8];
  bool equal;
  int64_t n_vectors;
  std::vector<int32_t> wtab;
};

static hp_status basis_facts(const std::vector<int64_t>& dims, BasisFacts* f, bool build_table) {
  f->nd = (int)dims.size();
  f->V = 1;
  f->K = 0;
  f->kmax = 0;
  f->Q = 1;
  for (int j = 0; j < 8; ++j) {
    f->L[j] = 1;
    f->ks[j] = 0;
    f->ps[j] = 1;
  }
  for (int j = 0; j < f->nd; ++j) {
    int L = (int)dims[j];
    int k = 0;
    while (L % 2 == 0) {
      L /= 2;
      ++k;
    }
    f->L[j] = (int)dims[j];
    f->ks[j] = k;
    f->ps[j] = L;
    f->K += k;
    if (k > f->kmax) f->kmax = k;
    f->Q *= L;
    f->V *= (int)dims[j];
  }
  int sizes[3] = {0, 0, 0};
  std::vector<int> colour(f->Q), rank(f->Q);
  for (int t = 0; t < f->Q; ++t) {
    int q[8], r = t;
    for (int j = 0; j < f->nd; ++j) {
      q[j] = r % f->ps[j];
      r /= f->ps[j];
    }
    colour[t] = three_colour(q, f->ps, f->nd);
    rank[t] = sizes[colour[t]]++;
  }
  f->equal = f->Q > 1 && sizes[0] == sizes[1] && sizes[1] == sizes[2];
  f->R = f->equal ? f->Q / 3 : 0;
  f->n_vectors = (f->Q == 1 || f->equal) ? (int64_t)f->V : ((int64_t)1 << f->K);
  int64_t P = 2;
  if (f->equal) {
    P = P * 3 / gcd64(P, 3);
    if (f->R > 1) P = P * f->R / gcd64(P, f->R);
  }
  if (P > 65535) {
    hp_set_error("period of the Fourier levels (%lld) does not fit 16 bits", (long long)P);
    return HP_EUNSUPPORTED;
  }
  f->P = (int)P;
  if (build_table) {
    f->wtab.resize(f->Q);
    for (int t = 0; t < f->Q; ++t) {
      int off = 0;
      for (int c = 0; c < colour[t]; ++c) off += sizes[c];
      f->wtab[t] = off + rank[t];
    }
  }
  return HP_OK;
}

extern "C" hp_status hp_basis_info(const hp_lattice* lat, hp_basis* out) {
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 8, &dims));
  if (!out) {
    hp_set_error("hp_basis_info: out is NULL");
    return HP_EINVAL;
  }
  BasisFacts f;
  HP_TRY(basis_facts(dims, &f, false));
  memset(out, 0, sizeof(*out));
  out->volume = f.V;
  out->n_vectors = f.n_vectors;
  out->K = f.K;
  out->Q = f.Q;
  out->R = f.R;
  out->period = f.P;
  out->kmax = f.kmax;
  for (int j = 0; j < 8; ++j) {
    out->ks[j] = f.ks[j];
    out->ps[j] = f.ps[j];
  }
  return HP_OK;
}

extern "C" hp_status hp_phase_values(int32_t period, double* out) {
  if (period < 1 || period > 65535 || !out) {
    hp_set_error("hp_phase_values: period in [1, 65535] and non-NULL output required");
    return HP_EINVAL;
  }
  for (int k = 0; k < period; ++k) phase_value(k, period, &out[2 * k], &out[2 * k + 1]);
  return HP_OK;
}

// ------------------------------------------------------- permutation kernel
// loc(x): for each level m = 1..kmax the m-th bits of the still-divisible
// dimensions (dimension 1 most significant) form an index i of a bits; the
// red-black position RB_a(i) = floor(i/2) + parity(i) 2^{a-1} (third lemma
// and theorem of Section 3.3) is appended below the earlier levels.  The
// odd block position w comes from the host table of the three-colouring.
__global__ void k_permutation(LatGeom g, uint32_t* __restrict__ loc) {
  const int stride = gridDim.x * blockDim.x;
  for (int site = blockIdx.x * blockDim.x + threadIdx.x; site < g.V; site += stride) {
    int x[8];
    int r = site;
    for (int j = 0; j < g.nd; ++j) {
      x[j] = r % g.L[j];
      r /= g.L[j];
    }
    uint32_t lb = 0;
    for (int m = 1; m <= g.kmax; ++m) {
      uint32_t idx = 0;
      int a = 0;
      for (int j = 0; j < g.nd; ++j) {
        if (m <= g.ks[j]) {
          idx = (idx << 1) | ((uint32_t)(x[j] >> (m - 1)) & 1u);
          ++a;
        }
      }
      uint32_t s = (idx >> 1) | ((uint32_t)(__popc(idx) & 1) << (a - 1));
      lb = (lb << a) | s;
    }
    uint32_t w = 0;
    if (g.Q > 1) {
      int t = 0;
      for (int j = 0; j < g.nd; ++j) t += (x[j] >> g.ks[j]) * g.qstride[j];
      w = (uint32_t)g.wtab[t];
    }
    loc[site] = lb * (uint32_t)g.Q + w;
  }
}

__global__ void k_probe_phases(LatGeom g, uint32_t first, int count, uint16_t* __restrict__ out) {
  const long long total = (long long)count * g.V;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
    int j = (int)(t / g.V);
    uint32_t site = (uint32_t)(t - (long long)j * g.V);
    out[t] = (uint16_t)probe_phase(g, site, first + (uint32_t)j);
  }
}

static int grid_for(hp_ctx* ctx, long long n, int threads) {
  long long b = (n + threads - 1) / threads;
  long long cap = (long long)ctx->num_sms * 16;
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

hp_status hp_get_lattice(hp_ctx* ctx, const std::vector<int64_t>& dims, LatticeSetup** out) {
  auto it = ctx->lattices.find(dims);
  if (it != ctx->lattices.end()) {
    *out = it->second.get();
    return HP_OK;
  }
  BasisFacts f;
  HP_TRY(basis_facts(dims, &f, true));
  std::unique_ptr<LatticeSetup> ls(new LatticeSetup());
  ls->dims = dims;
  ls->n_vectors = f.n_vectors;
  ls->equal = f.equal;
  LatGeom& g = ls->g;
  memset(&g, 0, sizeof(g));
  g.nd = f.nd;
  g.V = f.V;
  g.K = f.K;
  g.kmax = f.kmax;
  g.Q = f.Q;
  g.R = f.R;
  g.P = f.P;
  int qs = 1;
  for (int j = 0; j < 8; ++j) {
    g.L[j] = f.L[j];
    g.ks[j] = f.ks[j];
    g.qstride[j] = qs;
    qs *= f.ps[j];
  }
  std::vector<double2> tab(f.P);
  for (int k = 0; k < f.P; ++k) phase_value(k, f.P, &tab[k].x, &tab[k].y);
  cudaError_t e;
  e = cudaMalloc(&ls->loc.p, sizeof(uint32_t) * (size_t)f.V);
  if (e == cudaSuccess) e = cudaMalloc(&ls->wtab.p, sizeof(int32_t) * (size_t)f.Q);
  if (e == cudaSuccess) e = cudaMalloc(&ls->ptab.p, sizeof(double2) * (size_t)f.P);
  if (e != cudaSuccess) {
    cudaGetLastError();
    cudaFree(ls->loc.p);
    cudaFree(ls->wtab.p);
    cudaFree(ls->ptab.p);
    hp_set_error("lattice tables: cudaMalloc failed: %s", cudaGetErrorString(e));
    return HP_ENOMEM;
  }
  HP_CUDA(cudaMemcpyAsync(ls->wtab.p, f.wtab.data(), sizeof(int32_t) * f.Q, cudaMemcpyHostToDevice, ctx->stream));
  HP_CUDA(cudaMemcpyAsync(ls->ptab.p, tab.data(), sizeof(double2) * f.P, cudaMemcpyHostToDevice, ctx->stream));
  g.loc = (const uint32_t*)ls->loc.p;
  g.wtab = (const int32_t*)ls->wtab.p;
  g.ptab = (const double2*)ls->ptab.p;
  {
    ProfScope ps(ctx, "k_permutation");
    k_permutation<<<grid_for(ctx, f.V, 256), 256, 0, ctx->stream>>>(g, (uint32_t*)ls->loc.p);
  }
  HP_LAUNCH_CHECK();
  HP_CUDA(cudaStreamSynchronize(ctx->stream));   // host tables above must outlive the copies
  *out = ls.get();
  ctx->lattices[dims] = std::move(ls);
  return HP_OK;
}

extern "C" hp_status hp_permutation(hp_ctx* ctx, const hp_lattice* lat, uint32_t* loc_dev) {
  if (!ctx || !loc_dev) {
    hp_set_error("hp_permutation: NULL context or output");
    return HP_EINVAL;
  }
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 8, &dims));
  HP_CUDA(cudaSetDevice(ctx->device));
  LatticeSetup* ls = nullptr;
  HP_TRY(hp_get_lattice(ctx, dims, &ls));
  {
    ProfScope ps(ctx, "k_permutation");
    k_permutation<<<grid_for(ctx, ls->g.V, 256), 256, 0, ctx->stream>>>(ls->g, loc_dev);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}

extern "C" hp_status hp_probe_vectors(hp_ctx* ctx, const hp_lattice* lat, int64_t first, int64_t count,
                                      uint64_t z0_seed, uint16_t* phase_dev, int32_t* period_out) {
  return hp_probe_sequence(ctx, lat, HP_PROBE_HIERARCHICAL, first, count, z0_seed, phase_dev, period_out);
}

extern "C" hp_status hp_probe_sequence(hp_ctx* ctx, const hp_lattice* lat, int32_t kind, int64_t first,
                                       int64_t count, uint64_t z0_seed, uint16_t* phase_dev, int32_t* period_out) {
  if (!ctx) {
    hp_set_error("hp_probe_vectors: NULL context");
    return HP_EINVAL;
  }
  if (kind != HP_PROBE_HIERARCHICAL && kind != HP_PROBE_NATURAL && kind != HP_PROBE_Z2) {
    hp_set_error("unknown probe kind %d", kind);
    return HP_EINVAL;
  }
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 8, &dims));
  HP_CUDA(cudaSetDevice(ctx->device));
  LatticeSetup* ls = nullptr;
  HP_TRY(hp_get_lattice(ctx, dims, &ls));
  if (first < 0 || count < 0 || first + count > ls->g.V) {
    hp_set_error("probe range [%lld, %lld) outside [0, V = %d]", (long long)first, (long long)(first + count), ls->g.V);
    return HP_EINVAL;
  }
  if (kind == HP_PROBE_HIERARCHICAL && first + count > ls->n_vectors) {
    hp_set_error("only %lld nested vectors exist for this lattice (unequal odd colour classes)",
                 (long long)ls->n_vectors);
    return HP_EUNSUPPORTED;
  }
  if (kind == HP_PROBE_NATURAL && (ls->g.V & (ls->g.V - 1))) {
    hp_set_error("Hadamard vectors in natural order need V a power of two (V = %d)", ls->g.V);
    return HP_EUNSUPPORTED;
  }
  if (period_out) *period_out = ls->g.P;
  if (count == 0) return HP_OK;
  if (!phase_dev) {
    hp_set_error("hp_probe_vectors: phase_dev is NULL");
    return HP_EINVAL;
  }
  LatGeom g = ls->g;
  g.z0_seed = z0_seed;
  g.probe_kind = kind;
  {
    ProfScope ps(ctx, "k_probe_phases");
    k_probe_phases<<<grid_for(ctx, count * (long long)g.V, 256), 256, 0, ctx->stream>>>(g, (uint32_t)first,
                                                                                          (int)count, phase_dev);
  }
  HP_LAUNCH_CHECK();
  return HP_OK;
}
