// A Wilson stencil entry point that allocates nothing.
//
// Some callers cannot let a library allocate GPU memory: an application
// whose device memory is reserved up front by another framework's allocator
// (a cudaMalloc there fails or fragments the reserved pool), or one that
// must not add synchronising cudaMalloc / cudaFree calls to a latency-
// critical stream.  hp_operator_apply_noalloc serves them: the caller passes
// every input and output in device memory, and the only working memory is
// the fixed-size file-scope array below, which exists in every GPU that
// loads the library, until the process exits.
//
// The array holds the links of one lattice rearranged for coalesced loads
// (FP64, [mu][9 complex][V]); each call overwrites the part it uses before
// reading it, so nothing in it has to start at zero, but calls that overlap
// on the GPU (two streams, or two host threads) overwrite each other's links
// and race.
#include <algorithm>
#include <cstring>

#include "hp_fields.cuh"

#define HP_NOALLOC_MAX_SITES 20736   // 12^4; 36 double2 per site = 11.9 MB

static __device__ __align__(256) double2 g_noalloc_links[36 * HP_NOALLOC_MAX_SITES];

// Device address of g_noalloc_links on the current device.  Host code must not use the symbol
// itself (on the host it is only a stand-in); the address is looked up on every call, so a
// primary context that was torn down and re-created never leaves a stale pointer behind.
static hp_status noalloc_scratch(double2** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_links);
  if (e != cudaSuccess || !p) {
    hp_set_error("hp_operator_apply_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    return HP_ECUDA;
  }
  *out = (double2*)p;
  return HP_OK;
}

// canonical links complex128 [V][4][3][3] -> [mu][k][V] in the scratch array
__global__ void k_noalloc_links(const double2* __restrict__ in, int V, double2* __restrict__ out) {
  const long long total = 4LL * V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int site = (int)(t >> 2), mu = (int)(t & 3);
#pragma unroll
    for (int k = 0; k < 9; ++k) out[((size_t)mu * 9 + k) * V + site] = in[((size_t)site * 4 + mu) * 9 + k];
  }
}

__device__ __forceinline__ void canon_load(const double2* __restrict__ f, int V, int rhs, int site,
                                           cplx<double> (&s)[12]) {
  const double2* p = f + ((size_t)rhs * V + site) * 12;
#pragma unroll
  for (int k = 0; k < 12; ++k) {
    double2 v = __ldg(p + k);
    s[k] = {v.x, v.y};
  }
}

// out = D in on canonical complex128 [nrhs][V][4][3] fields, FP64 (same stencil arithmetic as
// the FP64 kernel of hp_operator_apply)
__global__ void k_noalloc_wilson(LatGeom g, const double2* __restrict__ in, double2* __restrict__ out, int nrhs) {
  const long long total = (long long)nrhs * g.V;
  for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const int rhs = (int)(t / g.V), site = (int)(t - (long long)rhs * g.V);
    int x[4], st[4];
    site_coords(g, site, x, st);
    cplx<double> acc[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = {0.0, 0.0};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
      const int L = g.L[mu];
      const int fw = (x[mu] + 1 == L) ? site - (L - 1) * st[mu] : site + st[mu];
      const int bw = (x[mu] == 0) ? site + (L - 1) * st[mu] : site - st[mu];
      cplx<double> psi[12], h[6], w[6], u[9];
      canon_load(in, g.V, rhs, fw, psi);
      LinkIO<PR64>::load(g, mu, site, u);
      if (mu == 0) project<0, -1>(psi, h);
      if (mu == 1) project<1, -1>(psi, h);
      if (mu == 2) project<2, -1>(psi, h);
      if (mu == 3) project<3, -1>(psi, h);
      su3_mul<double, false>(u, h, w);
      if (mu == 0) accumulate<0, -1>(acc, w);
      if (mu == 1) accumulate<1, -1>(acc, w);
      if (mu == 2) accumulate<2, -1>(acc, w);
      if (mu == 3) accumulate<3, -1>(acc, w);
      canon_load(in, g.V, rhs, bw, psi);
      LinkIO<PR64>::load(g, mu, bw, u);
      if (mu == 0) project<0, 1>(psi, h);
      if (mu == 1) project<1, 1>(psi, h);
      if (mu == 2) project<2, 1>(psi, h);
      if (mu == 3) project<3, 1>(psi, h);
      su3_mul<double, true>(u, h, w);
      if (mu == 0) accumulate<0, 1>(acc, w);
      if (mu == 1) accumulate<1, 1>(acc, w);
      if (mu == 2) accumulate<2, 1>(acc, w);
      if (mu == 3) accumulate<3, 1>(acc, w);
    }
    cplx<double> c[12];
    canon_load(in, g.V, rhs, site, c);
    const double diag = 1.0 + g.mass + (g.mass_field ? g.mass_field[site] : 0.0);
    double2* o = out + ((size_t)rhs * g.V + site) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = make_double2(diag * c[k].x - g.kappa * acc[k].x, diag * c[k].y - g.kappa * acc[k].y);
  }
}

// device that owns p, or -1 when p is not device (or managed) memory
static int owning_device(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

static bool ranges_overlap(const void* a, size_t na, const void* b, size_t nb) {
  const char *pa = (const char*)a, *pb = (const char*)b;
  return pa < pb + nb && pb < pa + na;
}

extern "C" hp_status hp_operator_apply_noalloc(const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                                               const double* in_dev, double* out_dev, void* cuda_stream) {
  if (!op || !lat || !in_dev || !out_dev || nrhs < 1) {
    hp_set_error("hp_operator_apply_noalloc: NULL argument or nrhs < 1");
    return HP_EINVAL;
  }
  if (op->kind != HP_OP_WILSON || !op->links) {
    hp_set_error("hp_operator_apply_noalloc: a Wilson operator with links is required");
    return HP_EINVAL;
  }
  if (op->csw != 0.0) {
    hp_set_error("hp_operator_apply_noalloc: plain Wilson only (csw = 0): the clover blocks need workspace");
    return HP_EINVAL;
  }
  if (lat->ndim < 1 || lat->ndim > 4) {
    hp_set_error("hp_operator_apply_noalloc: ndim = %d outside [1, 4]", lat->ndim);
    return HP_EINVAL;
  }
  long long V = 1;
  LatGeom g;
  memset(&g, 0, sizeof(g));
  g.nd = 4;
  for (int j = 0; j < 8; ++j) g.L[j] = 1;
  for (int j = 0; j < lat->ndim; ++j) {
    if (lat->dims[j] < 1 || lat->dims[j] > HP_NOALLOC_MAX_SITES) {
      hp_set_error("hp_operator_apply_noalloc: dims[%d] = %lld out of range", j, (long long)lat->dims[j]);
      return HP_EINVAL;
    }
    g.L[j] = (int)lat->dims[j];
    V *= lat->dims[j];
  }
  if (V > HP_NOALLOC_MAX_SITES) {
    hp_set_error("hp_operator_apply_noalloc: %lld sites exceed the fixed scratch of %d sites (12^4)", V,
                 HP_NOALLOC_MAX_SITES);
    return HP_EINVAL;
  }
  if (nrhs > 0x7fffffffLL || nrhs * V >= (1LL << 31)) {
    hp_set_error("hp_operator_apply_noalloc: nrhs * V must stay below 2^31");
    return HP_EINVAL;
  }
  const void* ptrs[4] = {op->links, in_dev, out_dev, op->mass_field};
  int owner[4] = {0, 0, 0, 0};
  for (int i = 0; i < 4; ++i) {
    if (!ptrs[i]) continue;
    owner[i] = owning_device(ptrs[i]);
    if (owner[i] < 0) {
      hp_set_error("hp_operator_apply_noalloc: links, mass field, input and output must be device memory");
      return HP_EINVAL;
    }
  }
  const size_t field = (size_t)nrhs * V * 24 * sizeof(double);
  if (ranges_overlap(out_dev, field, in_dev, field) ||
      ranges_overlap(out_dev, field, op->links, (size_t)V * 72 * sizeof(double)) ||
      (op->mass_field && ranges_overlap(out_dev, field, op->mass_field, (size_t)V * sizeof(double)))) {
    hp_set_error("hp_operator_apply_noalloc: the output overlaps the input, the links or the mass field");
    return HP_EINVAL;
  }
  int dev = -1;
  HP_CUDA(cudaGetDevice(&dev));
  for (int i = 0; i < 4; ++i) {
    if (ptrs[i] && owner[i] != dev) {
      hp_set_error("hp_operator_apply_noalloc: a buffer lives on device %d, the current device is %d", owner[i], dev);
      return HP_EINVAL;
    }
  }
  double2* scratch = nullptr;
  HP_TRY(noalloc_scratch(&scratch));
  g.V = (int)V;
  g.mass = op->mass;
  g.kappa = op->kappa;
  g.mass_field = op->mass_field;
  g.U64 = scratch;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int sms = 0;
  HP_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int thr = 128;
  long long nb = (4 * V + thr - 1) / thr;
  k_noalloc_links<<<(int)std::min<long long>(nb, sms * 8LL), thr, 0, s>>>((const double2*)op->links, (int)V, scratch);
  HP_LAUNCH_CHECK();
  nb = (nrhs * V + thr - 1) / thr;
  k_noalloc_wilson<<<(int)std::min<long long>(nb, sms * 16LL), thr, 0, s>>>(g, (const double2*)in_dev,
                                                                            (double2*)out_dev, (int)nrhs);
  HP_LAUNCH_CHECK();
  return HP_OK;
}
