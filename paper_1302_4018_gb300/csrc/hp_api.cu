// Entry points of the trace estimator: argument checks, operator
// preparation, the solve (slot scheduler), and the FP64 reductions of
// Section 1 / Section 2.2: q_m = sum_a v_{m,a}^H x_{m,a} and the prefix
// estimates T_s = (1/s) sum_{m<s} q_m.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>

#include "hp_internal.h"

hp_status hp_apply_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, const double* in,
                          double* out);
hp_status hp_apply_laplace(hp_ctx* ctx, LatGeom g, int nrhs, const double* in, double* out);
hp_status hp_wilson_deflation(hp_ctx* ctx, const LatGeom& g, int k, const double2* R, const double2* L,
                              const double* sigma, int64_t s_max, double2* q, double* exact_dev);
hp_status hp_wilson_deflation_gamma5(hp_ctx* ctx, const LatGeom& g, int k, const double2* W, const double* lam,
                                     int64_t s_max, double2* q, double* exact_dev);
hp_status hp_schur_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int nrhs, int prec, int eo_kernel,
                          const double* in, double* out);
hp_status hp_bench_wilson(hp_ctx* ctx, const hp_operator* op, LatGeom g, int prec, int nrhs, int iters, double* ms,
                          double* bytes, double* flops);

// q_m = sum_{a < dof} qj[m dof + a] (fixed order), then T_s = (1/s) sum_{m<s} q_m
// sequentially in FP64; probes m < first take q from q_prev.  Deflation adds the exact part
// sum_j 1/lambda_j (nlam eigenvalues lam) to every T_s.
__global__ void k_trace_prefix(const double2* __restrict__ qj, int dof, const double2* __restrict__ q_prev,
                               int first, int s_max, double2* __restrict__ q_out, double2* __restrict__ T,
                               const double* __restrict__ lam, int nlam, const double* __restrict__ exact0) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double exact = exact0 ? exact0[0] : 0.0;   // exact0: (re, im) of an exact part, or null
  const double exact_im = exact0 ? exact0[1] : 0.0;
  for (int j = 0; j < nlam; ++j) exact += 1.0 / lam[j];
  double2 acc = make_double2(0.0, 0.0);
  for (int m = 0; m < s_max; ++m) {
    double2 q;
    if (m < first) {
      q = q_prev[m];
    } else {
      q = make_double2(0.0, 0.0);
      const double2* p = qj + (size_t)(m - first) * dof;
      for (int a = 0; a < dof; ++a) {
        q.x += p[a].x;
        q.y += p[a].y;
      }
    }
    q_out[m] = q;
    acc.x += q.x;
    acc.y += q.y;
    T[m] = make_double2(exact + acc.x / (m + 1), exact_im + acc.y / (m + 1));
  }
}

// out(site) = scale * acc(site); sum over sites in a fixed tree order (one block)
__global__ void k_grad_finish(const double* __restrict__ acc, int V, double scale, double* __restrict__ out,
                              double* __restrict__ total) {
  __shared__ double sh[1024];
  double t = 0.0;
  for (int i = threadIdx.x; i < V; i += blockDim.x) {
    double v = scale * acc[i];
    out[i] = v;
    t += v;
  }
  sh[threadIdx.x] = t;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = sh[0];
}

static hp_status check_ctx(hp_ctx* ctx) {
  if (!ctx) {
    hp_set_error("NULL context");
    return HP_EINVAL;
  }
  HP_CUDA(cudaSetDevice(ctx->device));
  return HP_OK;
}

// geometry of an operator lattice: the user's dims for the probing basis, padded to 4-D for the stencil
static hp_status operator_geom(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, LatGeom* g,
                               LatticeSetup** setup) {
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 4, &dims));
  if (!op) {
    hp_set_error("operator is NULL");
    return HP_EINVAL;
  }
  if (op->kind != HP_OP_LAPLACIAN && op->kind != HP_OP_WILSON) {
    hp_set_error("unknown operator kind %d", op->kind);
    return HP_EINVAL;
  }
  if (!std::isfinite(op->mass) || !std::isfinite(op->kappa) || !std::isfinite(op->csw)) {
    hp_set_error("operator mass / kappa / csw not finite");
    return HP_EINVAL;
  }
  if (op->kind == HP_OP_LAPLACIAN && op->csw != 0.0) {
    hp_set_error("the clover term (csw != 0) belongs to the Wilson operator");
    return HP_EINVAL;
  }
  if (op->kind == HP_OP_WILSON && !op->links) {
    hp_set_error("Wilson operator needs links");
    return HP_EINVAL;
  }
  LatticeSetup* ls = nullptr;
  HP_TRY(hp_get_lattice(ctx, dims, &ls));
  *g = ls->g;
  g->nd = 4;
  for (int j = (int)dims.size(); j < 8; ++j) g->L[j] = 1;
  g->op_kind = op->kind;
  g->dof = op->kind == HP_OP_WILSON ? 12 : 1;
  g->parts = (op->kind == HP_OP_LAPLACIAN && g->P > 2) ? 2 : 1;
  if (setup) *setup = ls;
  return HP_OK;
}

static hp_status check_solver_args(int64_t s_max, double tol, const hp_solver_opts* opts, int64_t nvec, int64_t V) {
  if (!opts) {
    hp_set_error("solver options are NULL");
    return HP_EINVAL;
  }
  if (s_max < 1 || s_max > V) {
    hp_set_error("s_max = %lld outside [1, V = %lld]", (long long)s_max, (long long)V);
    return HP_EINVAL;
  }
  if (s_max > nvec) {
    hp_set_error("s_max = %lld exceeds the %lld nested vectors of this lattice", (long long)s_max, (long long)nvec);
    return HP_EUNSUPPORTED;
  }
  if (opts->first < 0 || opts->first >= s_max) {
    hp_set_error("first = %lld outside [0, s_max)", (long long)opts->first);
    return HP_EINVAL;
  }
  if (!(tol > 0.0) || !std::isfinite(tol)) {
    hp_set_error("tol must be a positive number");
    return HP_EINVAL;
  }
  if (opts->precision < HP_PREC_FP64 || opts->precision > HP_PREC_MIXED_BF16) {
    hp_set_error("unknown precision %d", opts->precision);
    return HP_EINVAL;
  }
  if (opts->rhs_block < 0 || opts->maxiter < 0) {
    hp_set_error("rhs_block and maxiter must be >= 0");
    return HP_EINVAL;
  }
  return HP_OK;
}

// the probing sequence of opts on lattice g: range checks and the geometry fields it needs
static hp_status set_probe_kind(const hp_solver_opts* opts, int64_t s_max, LatGeom* g) {
  g->z0_seed = opts->z0_seed;
  g->probe_kind = opts->probe_kind;
  if (opts->probe_kind == HP_PROBE_HIERARCHICAL) return HP_OK;
  if (opts->probe_kind != HP_PROBE_NATURAL && opts->probe_kind != HP_PROBE_Z2) {
    hp_set_error("unknown probe kind %d", opts->probe_kind);
    return HP_EINVAL;
  }
  if (opts->probe_kind == HP_PROBE_NATURAL && (g->V & (g->V - 1))) {
    hp_set_error("Hadamard vectors in natural order need V a power of two (V = %d)", g->V);
    return HP_EUNSUPPORTED;
  }
  if (s_max > g->V) {
    hp_set_error("s_max = %lld exceeds V = %d", (long long)s_max, g->V);
    return HP_EINVAL;
  }
  g->parts = 1;   // real +-1 vectors: one solve per vector for the Laplacian
  return HP_OK;
}

static int need_mask(int prec) {
  int m = 1 << PR64;
  if (prec == HP_PREC_MIXED_FP32) m |= 1 << PR32;
  if (prec == HP_PREC_MIXED_FP16 || prec == HP_PREC_MIXED_BF16) m |= (1 << PR16) | (1 << PR32);
  return m;
}

static hp_status prepare_operator(hp_ctx* ctx, const hp_operator* op, LatGeom* g, int prec, const char* tag) {
  HP_TRY(hp_prepare_mass(ctx, op, g, tag));
  if (op->kind == HP_OP_WILSON) HP_TRY(hp_prepare_wilson(ctx, op, g, tag, need_mask(prec)));
  return HP_OK;
}

static hp_status run_solve(hp_ctx* ctx, SolveProblem& pb, SolveResult& res) {
  // lattices of one problem share the operator family
  const int kind = pb.lats[0].op_kind;
  for (auto& g : pb.lats)
    if (g.op_kind != kind) {
      hp_set_error("a batch must use one operator kind");
      return HP_EINVAL;
    }
  return kind == HP_OP_WILSON ? hp_solve_wilson(ctx, pb, res) : hp_solve_laplace(ctx, pb, res);
}

// q and prefix of one lattice on the device, copied to the caller's host arrays
static hp_status finish_trace(hp_ctx* ctx, const SolveResult& res, int L, int dof, int64_t first, int64_t s_max,
                              double* q_inout, double* trace_prefix, const double* lam_dev = nullptr,
                              int nlam = 0) {
  void* p = nullptr;
  const size_t nq = res.qj[L].size();
  HP_TRY(hp_ws(ctx, "trace.qj", sizeof(double2) * std::max<size_t>(nq, 1), &p));
  double2* qj = (double2*)p;
  HP_TRY(hp_ws(ctx, "trace.qprev", sizeof(double2) * (size_t)s_max, &p));
  double2* qprev = (double2*)p;
  HP_TRY(hp_ws(ctx, "trace.qout", sizeof(double2) * (size_t)s_max, &p));
  double2* qout = (double2*)p;
  HP_TRY(hp_ws(ctx, "trace.T", sizeof(double2) * (size_t)s_max, &p));
  double2* T = (double2*)p;
  if (nq) HP_CUDA(cudaMemcpyAsync(qj, res.qj[L].data(), sizeof(double2) * nq, cudaMemcpyHostToDevice, ctx->stream));
  if (first > 0)
    HP_CUDA(cudaMemcpyAsync(qprev, q_inout, sizeof(double2) * (size_t)first, cudaMemcpyHostToDevice, ctx->stream));
  {
    ProfScope ps(ctx, "k_trace_prefix");
    k_trace_prefix<<<1, 32, 0, ctx->stream>>>(qj, dof, qprev, (int)first, (int)s_max, qout, T, lam_dev, nlam,
                                              nullptr);
  }
  HP_LAUNCH_CHECK();
  if (q_inout)
    HP_CUDA(cudaMemcpyAsync(q_inout, qout, sizeof(double2) * (size_t)s_max, cudaMemcpyDeviceToHost, ctx->stream));
  if (trace_prefix)
    HP_CUDA(cudaMemcpyAsync(trace_prefix, T, sizeof(double2) * (size_t)s_max, cudaMemcpyDeviceToHost, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

// quadrature-bracket stopping of the Laplacian CG (hp_trace_inv_bounds)
struct BoundsReq {
  double quad_tol, lambda_min;
  double *T_lower, *T_upper;
};

// solutions kept for the caller (hp_trace_inv_solutions)
struct KeepReq {
  int64_t n_keep;
  double* x_out;   // device, complex [n_keep][V][12]
};

// deflated probing of the Laplacian (hp_trace_inv_deflated)
struct DeflReq {
  int32_t k;
  const double* evecs;   // [k][V], host or device
  const double* evals;   // [k], host
};

static hp_status trace_common(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max, double tol,
                              const hp_solver_opts* opts, double* q_inout, double* trace_prefix, double* dT_dmu,
                              double* dT_dm, hp_solve_stats* stats, const BoundsReq* bounds = nullptr,
                              const DeflReq* defl = nullptr, const KeepReq* keep = nullptr) {
  HP_TRY(check_ctx(ctx));
  LatGeom g;
  LatticeSetup* ls = nullptr;
  HP_TRY(operator_geom(ctx, op, lat, &g, &ls));
  HP_TRY(check_solver_args(s_max, tol, opts, opts->probe_kind ? g.V : ls->n_vectors, g.V));
  HP_TRY(set_probe_kind(opts, s_max, &g));
  if (!trace_prefix) {
    hp_set_error("trace_prefix is NULL");
    return HP_EINVAL;
  }
  if (opts->first > 0 && !q_inout) {
    hp_set_error("first > 0 needs the earlier quadratures in q_inout");
    return HP_EINVAL;
  }
  const bool grad = dT_dmu != nullptr;
  if (grad && opts->first != 0) {
    hp_set_error("the gradient needs first == 0");
    return HP_EINVAL;
  }
  if (opts->dilution != 0 && opts->dilution != (op->kind == HP_OP_WILSON ? 12 : 1)) {
    hp_set_error("dilution %d not supported (Wilson: 12, Laplacian: 1)", opts->dilution);
    return HP_EINVAL;
  }
  HP_TRY(prepare_operator(ctx, op, &g, opts->precision, "op0"));
  const double* lam_dev = nullptr;
  if (defl) {
    const void* p = nullptr;
    HP_TRY(hp_device_view(ctx, defl->evecs, sizeof(double) * (size_t)defl->k * g.V, "defl.V", &p));
    g.defl_V = (const double*)p;
    g.defl_k = defl->k;
    void* l = nullptr;
    HP_TRY(hp_ws(ctx, "defl.lam", sizeof(double) * (size_t)defl->k, &l));
    HP_CUDA(cudaMemcpyAsync(l, defl->evals, sizeof(double) * (size_t)defl->k, cudaMemcpyHostToDevice, ctx->stream));
    lam_dev = (const double*)l;
  }
  if (bounds) {   // Gauss-Radau node: the caller's bound, else m + min mu(x) (the Laplacian part is PSD)
    double mu = bounds->lambda_min;
    if (!(mu > 0.0)) {
      mu = op->mass;
      if (op->mass_field) {
        std::vector<double> mf((size_t)g.V);
        HP_CUDA(cudaMemcpyAsync(mf.data(), g.mass_field, sizeof(double) * mf.size(), cudaMemcpyDeviceToHost,
                                ctx->stream));
        HP_CUDA(cudaStreamSynchronize(ctx->stream));
        mu += *std::min_element(mf.begin(), mf.end());
      }
    }
    if (!(mu > 0.0) || !std::isfinite(mu)) {
      hp_set_error("the Gauss-Radau node must be positive (lambda_min = %g): the operator is not positive definite",
                   mu);
      return HP_EINVAL;
    }
    g.quad_mu = mu;
    g.quad_tol = bounds->quad_tol;
  }
  SolveProblem pb;
  pb.lats.push_back(g);
  pb.s_max.push_back(s_max);
  pb.first.push_back(opts->first);
  pb.tol = tol;
  pb.opts = *opts;
  pb.want_grad = grad;
  if (keep) {
    if (op->kind != HP_OP_WILSON) {
      hp_set_error("solutions are kept for the Wilson operator only");
      return HP_EINVAL;
    }
    if (keep->n_keep < 0 || keep->n_keep > (s_max - opts->first) * 12) {
      hp_set_error("n_keep = %lld outside [0, 12 (s_max - first)]", (long long)keep->n_keep);
      return HP_EINVAL;
    }
    if (keep->n_keep > 0) {
      if (!keep->x_out || !hp_is_device_ptr(keep->x_out)) {
        hp_set_error("x_out must be device memory");
        return HP_EINVAL;
      }
      pb.x_keep = (double2*)keep->x_out;
      pb.n_keep = keep->n_keep;
    }
  }
  if (grad) {
    void* p = nullptr;
    HP_TRY(hp_ws(ctx, "grad.acc", sizeof(double) * (size_t)g.V, &p));
    HP_CUDA(cudaMemsetAsync(p, 0, sizeof(double) * (size_t)g.V, ctx->stream));
    pb.grad_dev.push_back((double*)p);
  }
  SolveResult res;
  HP_TRY(run_solve(ctx, pb, res));
  const int dof = op->kind == HP_OP_WILSON ? 12 : g.parts;
  HP_TRY(finish_trace(ctx, res, 0, dof, opts->first, s_max, q_inout, trace_prefix, lam_dev,
                      defl ? defl->k : 0));
  if (bounds) {   // T_s bounds: (1/s) sum over probes and parts of the per-solve brackets
    double lo = 0.0, hi = 0.0;
    for (int64_t m = 0; m < s_max; ++m) {
      for (int a = 0; a < dof; ++a) {
        const double2 b = res.qb[0][(size_t)m * dof + a];
        lo += b.x;
        hi += b.y;
      }
      bounds->T_lower[m] = lo / (double)(m + 1);
      bounds->T_upper[m] = hi / (double)(m + 1);
    }
  }
  if (grad) {
    void* p = nullptr;
    double* out = dT_dmu;
    bool host_out = !hp_is_device_ptr(dT_dmu);
    if (host_out) {
      HP_TRY(hp_ws(ctx, "grad.out", sizeof(double) * (size_t)g.V, &p));
      out = (double*)p;
    }
    HP_TRY(hp_ws(ctx, "grad.total", sizeof(double), &p));
    double* tot = (double*)p;
    {
      ProfScope ps(ctx, "k_grad_finish");
      k_grad_finish<<<1, 1024, 0, ctx->stream>>>(pb.grad_dev[0], g.V, -1.0 / (double)s_max, out, tot);
    }
    HP_LAUNCH_CHECK();
    if (host_out) HP_CUDA(cudaMemcpyAsync(dT_dmu, out, sizeof(double) * (size_t)g.V, cudaMemcpyDeviceToHost, ctx->stream));
    double t = 0.0;
    HP_CUDA(cudaMemcpyAsync(&t, tot, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    if (dT_dm) *dT_dm = t;
  }
  if (stats) *stats = res.stats;
  if (res.unconverged) {
    hp_set_error("%d right-hand sides missed tol within maxiter", res.stats.n_unconverged);
    return HP_ENOCONV;
  }
  return HP_OK;
}

extern "C" hp_status hp_trace_inv(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max, double tol,
                                  const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                                  hp_solve_stats* stats) {
  return trace_common(ctx, op, lat, s_max, tol, opts, q_inout, trace_prefix, nullptr, nullptr, stats);
}

extern "C" hp_status hp_trace_inv_solutions(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                                            double tol, const hp_solver_opts* opts, int64_t n_keep, double* x_out,
                                            double* q_inout, double* trace_prefix, hp_solve_stats* stats) {
  const KeepReq keep{n_keep, x_out};
  return trace_common(ctx, op, lat, s_max, tol, opts, q_inout, trace_prefix, nullptr, nullptr, stats, nullptr, nullptr,
                      &keep);
}

extern "C" hp_status hp_trace_prefix(hp_ctx* ctx, int64_t s_max, const double* q, double* trace_prefix) {
  HP_TRY(check_ctx(ctx));
  if (s_max < 1 || s_max >= (1LL << 31) || !q || !trace_prefix) {
    hp_set_error("hp_trace_prefix: s_max = %lld outside [1, 2^31) or a NULL array", (long long)s_max);
    return HP_EINVAL;
  }
  // every q_m is an input (first = s_max): the kernel and summation order of hp_trace_inv
  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "trace.qprev", sizeof(double2) * (size_t)s_max, &p));
  double2* qprev = (double2*)p;
  HP_TRY(hp_ws(ctx, "trace.qout", sizeof(double2) * (size_t)s_max, &p));
  double2* qout = (double2*)p;
  HP_TRY(hp_ws(ctx, "trace.T", sizeof(double2) * (size_t)s_max, &p));
  double2* T = (double2*)p;
  HP_CUDA(cudaMemcpyAsync(qprev, q, sizeof(double2) * (size_t)s_max, cudaMemcpyDefault, ctx->stream));
  {
    ProfScope ps(ctx, "k_trace_prefix");
    k_trace_prefix<<<1, 32, 0, ctx->stream>>>(nullptr, 0, qprev, (int)s_max, (int)s_max, qout, T, nullptr, 0,
                                              nullptr);
  }
  HP_LAUNCH_CHECK();
  HP_CUDA(cudaMemcpyAsync(trace_prefix, T, sizeof(double2) * (size_t)s_max, cudaMemcpyDefault, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

// deflated probing of the Wilson matrix: the plain solves, then the deflation correction of each
// quadrature and the exact part on the device (hp_wdefl.cu).  left = NULL: evecs / evals are
// eigenpairs of gamma_5 D; else evecs / left / evals are singular triplets D v = sigma u.
static hp_status trace_deflated_wilson(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                       const double* evecs, const double* left, const double* evals, int64_t s_max,
                                       double tol, const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                                       hp_solve_stats* stats) {
  HP_TRY(check_ctx(ctx));
  LatGeom g;
  HP_TRY(operator_geom(ctx, op, lat, &g, nullptr));
  if (!opts || !trace_prefix) {
    hp_set_error("deflation: solver options and trace_prefix required");
    return HP_EINVAL;
  }
  HP_TRY(set_probe_kind(opts, s_max, &g));
  if (opts->probe_kind != HP_PROBE_HIERARCHICAL) {
    hp_set_error("deflated Wilson probing uses the hierarchical vectors (probe_kind 0)");
    return HP_EUNSUPPORTED;
  }
  if (k < 1 || (int64_t)k > std::min<int64_t>(12LL * g.V, 65535) || !evecs || !evals) {
    hp_set_error("deflation: 1 <= k <= min(12 V, 65535) and non-NULL eigenvectors and eigenvalues required (k = %d)",
                 k);
    return HP_EINVAL;
  }
  for (int j = 0; j < k; ++j)
    if ((left ? !(evals[j] > 0.0) : !(evals[j] != 0.0)) || !std::isfinite(evals[j])) {
      hp_set_error(left ? "deflation: singular value %d is %g" : "deflation: eigenvalue %d of gamma_5 D is %g", j,
                   evals[j]);
      return HP_EINVAL;
    }
  std::vector<double> qraw(2 * (size_t)s_max, 0.0), Traw(2 * (size_t)s_max, 0.0);
  HP_TRY(trace_common(ctx, op, lat, s_max, tol, opts, qraw.data(), Traw.data(), nullptr, nullptr, stats));
  const void* p = nullptr;
  HP_TRY(hp_device_view(ctx, evecs, sizeof(double2) * 12 * (size_t)k * g.V, "wdefl.W", &p));
  const double2* W = (const double2*)p;
  const double2* Ld = nullptr;
  if (left) {
    HP_TRY(hp_device_view(ctx, left, sizeof(double2) * 12 * (size_t)k * g.V, "wdefl.Lin", &p));
    Ld = (const double2*)p;
  }
  void* v = nullptr;
  HP_TRY(hp_ws(ctx, "wdefl.lam", sizeof(double) * (size_t)k, &v));
  double* lam = (double*)v;
  HP_CUDA(cudaMemcpyAsync(lam, evals, sizeof(double) * (size_t)k, cudaMemcpyHostToDevice, ctx->stream));
  HP_TRY(hp_ws(ctx, "wdefl.exact", 2 * sizeof(double), &v));
  double* exact = (double*)v;
  HP_TRY(hp_ws(ctx, "trace.qprev", sizeof(double2) * (size_t)s_max, &v));
  double2* qprev = (double2*)v;
  HP_TRY(hp_ws(ctx, "trace.qout", sizeof(double2) * (size_t)s_max, &v));
  double2* qout = (double2*)v;
  HP_TRY(hp_ws(ctx, "trace.T", sizeof(double2) * (size_t)s_max, &v));
  double2* T = (double2*)v;
  HP_CUDA(cudaMemcpyAsync(qprev, qraw.data(), sizeof(double2) * (size_t)s_max, cudaMemcpyHostToDevice, ctx->stream));
  if (left) HP_TRY(hp_wilson_deflation(ctx, g, k, W, Ld, lam, s_max, qprev, exact));
  else HP_TRY(hp_wilson_deflation_gamma5(ctx, g, k, W, lam, s_max, qprev, exact));
  {
    ProfScope ps(ctx, "k_trace_prefix");
    k_trace_prefix<<<1, 32, 0, ctx->stream>>>(nullptr, 0, qprev, (int)s_max, (int)s_max, qout, T, nullptr, 0, exact);
  }
  HP_LAUNCH_CHECK();
  if (q_inout)
    HP_CUDA(cudaMemcpyAsync(q_inout, qout, sizeof(double2) * (size_t)s_max, cudaMemcpyDefault, ctx->stream));
  HP_CUDA(cudaMemcpyAsync(trace_prefix, T, sizeof(double2) * (size_t)s_max, cudaMemcpyDefault, ctx->stream));
  HP_CUDA(cudaStreamSynchronize(ctx->stream));
  return HP_OK;
}

extern "C" hp_status hp_trace_inv_deflated(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                           const double* evecs, const double* evals, int64_t s_max, double tol,
                                           const hp_solver_opts* opts, double* q_inout, double* trace_prefix,
                                           hp_solve_stats* stats) {
  if (op && op->kind == HP_OP_WILSON) {
    if (opts && opts->first != 0) {
      hp_set_error("deflated probing needs first == 0");
      return HP_EINVAL;
    }
    return trace_deflated_wilson(ctx, op, lat, k, evecs, nullptr, evals, s_max, tol, opts, q_inout, trace_prefix,
                                 stats);
  }
  if (!op || op->kind != HP_OP_LAPLACIAN) {
    hp_set_error("deflated probing needs a Laplacian or Wilson operator");
    return HP_EINVAL;
  }
  std::vector<int64_t> dims;
  HP_TRY(hp_validate_lattice(lat, 4, &dims));
  int64_t V = 1;
  for (int64_t d : dims) V *= d;
  if (k < 1 || k > V || !evecs || !evals) {
    hp_set_error("deflation: 1 <= k <= V and non-NULL eigenvectors and eigenvalues required (k = %d)", k);
    return HP_EINVAL;
  }
  for (int j = 0; j < k; ++j)
    if (!(evals[j] > 0.0) || !std::isfinite(evals[j])) {
      hp_set_error("deflation: eigenvalue %d is %g (the Laplacian is positive definite)", j, evals[j]);
      return HP_EINVAL;
    }
  if (opts && opts->first != 0) {
    hp_set_error("deflated probing needs first == 0");
    return HP_EINVAL;
  }
  const DeflReq d{k, evecs, evals};
  return trace_common(ctx, op, lat, s_max, tol, opts, q_inout, trace_prefix, nullptr, nullptr, stats, nullptr, &d);
}

extern "C" hp_status hp_trace_inv_deflated_svd(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t k,
                                               const double* right, const double* left, const double* sigma,
                                               int64_t s_max, double tol, const hp_solver_opts* opts, double* q_inout,
                                               double* trace_prefix, hp_solve_stats* stats) {
  if (!op || op->kind != HP_OP_WILSON) {
    hp_set_error("deflation with singular triplets serves the Wilson operator");
    return HP_EINVAL;
  }
  if (!left) {
    hp_set_error("deflation with singular triplets: left vectors required");
    return HP_EINVAL;
  }
  if (opts && opts->first != 0) {
    hp_set_error("deflated probing needs first == 0");
    return HP_EINVAL;
  }
  return trace_deflated_wilson(ctx, op, lat, k, right, left, sigma, s_max, tol, opts, q_inout, trace_prefix, stats);
}

extern "C" hp_status hp_trace_inv_sparse(hp_ctx* ctx, int32_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                         const double* values, const int32_t* paths, const int32_t* radices,
                                         int32_t n_levels, int64_t s_max, double tol, const hp_solver_opts* opts,
                                         double* q_inout, double* trace_prefix, hp_solve_stats* stats) {
  HP_TRY(check_ctx(ctx));
  if (!values) {
    hp_set_error("sparse matrix: values are NULL");
    return HP_EINVAL;
  }
  HP_TRY(check_solver_args(s_max, tol, opts, n, n));
  if (opts->precision != HP_PREC_FP64 && opts->precision != HP_PREC_MIXED_FP32) {
    hp_set_error("the sparse CG iterates in FP64 or FP32 (precision %d)", opts->precision);
    return HP_EUNSUPPORTED;
  }
  if (opts->dilution != 0 && opts->dilution != 1) {
    hp_set_error("dilution %d not supported for a sparse matrix (1)", opts->dilution);
    return HP_EINVAL;
  }
  if (!trace_prefix || (opts->first > 0 && !q_inout)) {
    hp_set_error("trace_prefix is NULL, or first > 0 without the earlier quadratures in q_inout");
    return HP_EINVAL;
  }
  LatGeom g;
  HP_TRY(hp_sparse_geom(ctx, n, row_ptr, col_idx, values, paths, radices, n_levels, s_max, opts->probe_kind, &g));
  g.z0_seed = opts->z0_seed;
  SolveProblem pb;
  pb.lats.push_back(g);
  pb.s_max.push_back(s_max);
  pb.first.push_back(opts->first);
  pb.tol = tol;
  pb.opts = *opts;
  SolveResult res;
  HP_TRY(hp_solve_laplace(ctx, pb, res));
  HP_TRY(finish_trace(ctx, res, 0, g.parts, opts->first, s_max, q_inout, trace_prefix));
  if (stats) *stats = res.stats;
  if (res.unconverged) {
    hp_set_error("%d right-hand sides missed tol within maxiter", res.stats.n_unconverged);
    return HP_ENOCONV;
  }
  return HP_OK;
}

extern "C" hp_status hp_trace_inv_bounds(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                                         double quad_tol, double lambda_min, const hp_solver_opts* opts,
                                         double* trace_prefix, double* T_lower, double* T_upper,
                                         hp_solve_stats* stats) {
  if (!op || op->kind != HP_OP_LAPLACIAN) {
    hp_set_error("hp_trace_inv_bounds: the quadrature bounds need a Hermitian positive definite operator "
                 "(the Laplacian)");
    return HP_EINVAL;
  }
  if (!T_lower || !T_upper || !(quad_tol > 0.0) || !std::isfinite(quad_tol)) {
    hp_set_error("hp_trace_inv_bounds: T_lower, T_upper and a positive quad_tol are required");
    return HP_EINVAL;
  }
  if (opts && opts->first != 0) {
    hp_set_error("hp_trace_inv_bounds: first must be 0");
    return HP_EINVAL;
  }
  const BoundsReq b{quad_tol, lambda_min, T_lower, T_upper};
  return trace_common(ctx, op, lat, s_max, quad_tol, opts, nullptr, trace_prefix, nullptr, nullptr, stats, &b);
}

extern "C" hp_status hp_trace_inv_grad(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t s_max,
                                       double tol, const hp_solver_opts* opts, double* trace_prefix, double* dT_dmu,
                                       double* dT_dm, hp_solve_stats* stats) {
  if (!dT_dmu) {
    hp_set_error("dT_dmu is NULL");
    return HP_EINVAL;
  }
  return trace_common(ctx, op, lat, s_max, tol, opts, nullptr, trace_prefix, dT_dmu, dT_dm, stats);
}

extern "C" hp_status hp_trace_inv_batch(hp_ctx* ctx, int32_t nlat, const hp_operator* ops, const hp_lattice* lats,
                                        const int64_t* s_max, double tol, const hp_solver_opts* opts,
                                        double* const* trace_prefix, hp_solve_stats* stats) {
  HP_TRY(check_ctx(ctx));
  if (nlat < 1 || !ops || !lats || !s_max || !trace_prefix) {
    hp_set_error("hp_trace_inv_batch: empty batch or NULL array");
    return HP_EINVAL;
  }
  if (!opts || opts->first != 0) {
    hp_set_error("hp_trace_inv_batch: options must be given with first == 0");
    return HP_EINVAL;
  }
  SolveProblem pb;
  pb.tol = tol;
  pb.opts = *opts;
  for (int i = 0; i < nlat; ++i) {
    LatGeom g;
    LatticeSetup* ls = nullptr;
    HP_TRY(operator_geom(ctx, &ops[i], &lats[i], &g, &ls));
    HP_TRY(check_solver_args(s_max[i], tol, opts, opts->probe_kind ? g.V : ls->n_vectors, g.V));
    HP_TRY(set_probe_kind(opts, s_max[i], &g));
    if (!trace_prefix[i]) {
      hp_set_error("trace_prefix[%d] is NULL", i);
      return HP_EINVAL;
    }
    char tag[32];
    snprintf(tag, sizeof(tag), "op%d", i);
    HP_TRY(prepare_operator(ctx, &ops[i], &g, opts->precision, tag));
    pb.lats.push_back(g);
    pb.s_max.push_back(s_max[i]);
    pb.first.push_back(0);
  }
  SolveResult res;
  HP_TRY(run_solve(ctx, pb, res));
  for (int i = 0; i < nlat; ++i) {
    const int dof = ops[i].kind == HP_OP_WILSON ? 12 : pb.lats[i].parts;
    HP_TRY(finish_trace(ctx, res, i, dof, 0, s_max[i], nullptr, trace_prefix[i]));
  }
  if (stats) *stats = res.stats;
  if (res.unconverged) {
    hp_set_error("%d right-hand sides missed tol within maxiter", res.stats.n_unconverged);
    return HP_ENOCONV;
  }
  return HP_OK;
}

extern "C" hp_status hp_operator_apply(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                                       int32_t precision, const double* in, double* out) {
  HP_TRY(check_ctx(ctx));
  LatGeom g;
  HP_TRY(operator_geom(ctx, op, lat, &g, nullptr));
  if (nrhs < 1 || nrhs > 65535 || !in || !out) {
    hp_set_error("hp_operator_apply: nrhs in [1, 65535] and non-NULL buffers required");
    return HP_EINVAL;
  }
  if (precision < HP_PREC_FP64 || precision > HP_PREC_MIXED_BF16) {
    hp_set_error("unknown precision %d", precision);
    return HP_EINVAL;
  }
  if (op->kind == HP_OP_LAPLACIAN) {
    HP_TRY(hp_prepare_mass(ctx, op, &g, "apply"));
    return hp_apply_laplace(ctx, g, (int)nrhs, in, out);
  }
  return hp_apply_wilson(ctx, op, g, (int)nrhs, precision, in, out);
}

extern "C" hp_status hp_schur_apply(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int64_t nrhs,
                                    int32_t precision, int32_t eo_kernel, const double* in, double* out) {
  HP_TRY(check_ctx(ctx));
  LatGeom g;
  HP_TRY(operator_geom(ctx, op, lat, &g, nullptr));
  if (op->kind != HP_OP_WILSON) {
    hp_set_error("hp_schur_apply: the even-odd Schur complement belongs to the Wilson operator");
    return HP_EINVAL;
  }
  if (nrhs < 1 || nrhs > 65532 || !in || !out) {
    hp_set_error("hp_schur_apply: nrhs in [1, 65532] and non-NULL buffers required");
    return HP_EINVAL;
  }
  if (precision < HP_PREC_FP64 || precision > HP_PREC_MIXED_BF16) {
    hp_set_error("unknown precision %d", precision);
    return HP_EINVAL;
  }
  return hp_schur_wilson(ctx, op, g, (int)nrhs, precision, eo_kernel, in, out);
}

extern "C" hp_status hp_dslash_bench(hp_ctx* ctx, const hp_operator* op, const hp_lattice* lat, int32_t precision,
                                     int32_t nrhs, int32_t iters, double* ms_per_launch, double* bytes_per_launch,
                                     double* flops_per_launch) {
  HP_TRY(check_ctx(ctx));
  LatGeom g;
  HP_TRY(operator_geom(ctx, op, lat, &g, nullptr));
  if (op->kind != HP_OP_WILSON || nrhs < 1 || nrhs > 65535 || iters < 1 || !ms_per_launch || !bytes_per_launch ||
      !flops_per_launch) {
    hp_set_error("hp_dslash_bench: Wilson operator, nrhs >= 1, iters >= 1 and outputs required");
    return HP_EINVAL;
  }
  if (precision < HP_PREC_FP64 || precision > HP_PREC_MIXED_BF16) {
    hp_set_error("unknown precision %d", precision);
    return HP_EINVAL;
  }
  return hp_bench_wilson(ctx, op, g, precision, nrhs, iters, ms_per_launch, bytes_per_launch, flops_per_launch);
}
