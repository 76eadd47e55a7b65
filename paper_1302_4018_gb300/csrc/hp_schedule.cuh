// Slot scheduler shared by the Wilson and Laplacian solvers.
//
// The right-hand sides of every lattice of a problem form one queue
// (lattice, probe m, dilution index / part a).  A fixed set of solver
// slots works through it: every kernel launch advances all occupied slots
// (grid.x = slot), converged slots are harvested (quadrature, gradient) and
// refilled with the next right-hand side, so lattices of different sizes
// and convergence speeds share every launch.  The host only looks at the
// per-slot status every `check_every` iterations; the iteration itself is
// driven by device-side scalars and masks (and can be replayed from a
// captured CUDA graph).
#pragma once
#include <chrono>
#include <vector>

template <class Engine>
hp_status run_schedule(hp_ctx* ctx, Engine& eng, SolveProblem& pb, SolveResult& res, int dof_wilson, double delta) {
  auto t0 = std::chrono::steady_clock::now();
  const int nl = (int)pb.lats.size();
  int Vmax = 0;
  for (auto& g : pb.lats) Vmax = std::max(Vmax, g.V);

  struct Item {
    int lat, m, a;
  };
  std::vector<Item> queue;
  res.qj.assign(nl, {});
  res.qb.assign(nl, {});
  for (int L = 0; L < nl; ++L) {
    const int dof = pb.lats[L].op_kind == HP_OP_WILSON ? dof_wilson : pb.lats[L].parts;
    const int64_t n = (pb.s_max[L] - pb.first[L]) * dof;
    res.qj[L].assign((size_t)n, make_double2(0.0, 0.0));
    res.qb[L].assign((size_t)n, make_double2(0.0, 0.0));
    for (int64_t m = pb.first[L]; m < pb.s_max[L]; ++m)
      for (int a = 0; a < dof; ++a) queue.push_back({L, (int)m, a});
  }
  int nslots = pb.opts.rhs_block;
  if (nslots <= 0) {
    long long want = (4LL << 20) / std::max(1, Vmax);
    nslots = (int)std::max(12LL, std::min(want, 256LL));
  }
  nslots = (int)std::min<long long>(nslots, std::max<size_t>(1, queue.size()));
  nslots = std::min(nslots, 65535);   // one grid dimension of the solver kernels
  nslots = (nslots + Engine::GROUP_MAX - 1) / Engine::GROUP_MAX * Engine::GROUP_MAX;
  int big = 0;
  for (int L = 1; L < nl; ++L)
    if (pb.lats[L].V > pb.lats[big].V) big = L;

  void* p = nullptr;
  HP_TRY(hp_ws(ctx, "solve.lats", sizeof(LatGeom) * nl, &p));
  LatGeom* lats_dev = (LatGeom*)p;
  HP_CUDA(cudaMemcpyAsync(lats_dev, pb.lats.data(), sizeof(LatGeom) * nl, cudaMemcpyHostToDevice, ctx->stream));
  HP_TRY(hp_ws(ctx, "solve.state", sizeof(SlotState) * nslots, &p));
  SlotState* st_dev = (SlotState*)p;
  HP_TRY(hp_ws(ctx, "solve.slots", sizeof(int) * nslots, &p));
  int* dev_slots = (int*)p;
  std::vector<SlotState> host(nslots);
  memset(host.data(), 0, sizeof(SlotState) * nslots);
  eng.big_lat = big;
  eng.one_lat = nl == 1;
  HP_TRY(eng.setup(nslots, Vmax, lats_dev, st_dev, pb.opts, pb.tol, delta, pb.lats[big]));
  const int G = eng.group();   // slots refilled together (one lattice per group: the stencil shares links)

  const int chunk = pb.opts.check_every > 0 ? pb.opts.check_every : 8;
  const bool use_graph = pb.opts.use_graph && !ctx->profiling;
  cudaGraphExec_t gexec = nullptr;
  if (use_graph) {
    cudaGraph_t graph = nullptr;
    HP_CUDA(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    hp_status s = HP_OK;
    for (int c = 0; c < chunk && s == HP_OK; ++c) s = eng.iteration();
    cudaError_t e = cudaStreamEndCapture(ctx->stream, &graph);
    if (s != HP_OK) return s;
    if (e != cudaSuccess) {
      hp_set_error("graph capture failed: %s", cudaGetErrorString(e));
      return HP_ECUDA;
    }
    e = cudaGraphInstantiate(&gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      hp_set_error("graph instantiate failed: %s", cudaGetErrorString(e));
      return HP_ECUDA;
    }
  }

  memset(&res.stats, 0, sizeof(res.stats));
  res.stats.iterations_min = 0x7fffffff;
  size_t qpos = 0;
  hp_status status = HP_OK;
  while (true) {
    bool any_init = false, any_run = false;
    for (int g0 = 0; g0 < nslots; g0 += G) {
      // the slots of a group hold right-hand sides of one lattice: an empty slot whose partners are
      // still running takes the next item only if it belongs to their lattice (the queue runs
      // through the lattices in order, so otherwise none of theirs is left)
      int L = -1;
      for (int r = 0; r < G; ++r)
        if (host[g0 + r].status != SLOT_EMPTY) L = host[g0 + r].lat;
      for (int r = 0; r < G && qpos < queue.size(); ++r) {
        SlotState& S = host[g0 + r];
        if (S.status != SLOT_EMPTY) continue;
        if (L >= 0 && queue[qpos].lat != L) break;
        L = queue[qpos].lat;
        const Item& it = queue[qpos++];
        memset(&S, 0, sizeof(SlotState));
        S.status = SLOT_INIT;
        S.lat = it.lat;
        S.m = it.m;
        S.a = it.a;
        any_init = true;
      }
    }
    for (int sl = 0; sl < nslots; ++sl)
      if (host[sl].status == SLOT_RUN) any_run = true;
    HP_CUDA(cudaMemcpyAsync(st_dev, host.data(), sizeof(SlotState) * nslots, cudaMemcpyHostToDevice, ctx->stream));
    if (any_init) HP_TRY(eng.init());
    if (!any_init && !any_run) break;
    if (use_graph) {
      HP_CUDA(cudaGraphLaunch(gexec, ctx->stream));
      ctx->launches += (long long)chunk * eng.kernels_per_iteration();
    } else {
      for (int c = 0; c < chunk; ++c) HP_TRY(eng.iteration());
    }
    HP_CUDA(cudaMemcpyAsync(host.data(), st_dev, sizeof(SlotState) * nslots, cudaMemcpyDeviceToHost, ctx->stream));
    HP_CUDA(cudaStreamSynchronize(ctx->stream));
    std::vector<int> done;
    for (int sl = 0; sl < nslots; ++sl)
      if (host[sl].status == SLOT_DONE || host[sl].status == SLOT_FAIL) done.push_back(sl);
    if (!done.empty()) {
      HP_TRY(eng.harvest(done, pb, dev_slots));
      if (pb.x_keep) HP_TRY(eng.keep(done, host, pb));
      HP_CUDA(cudaMemcpyAsync(host.data(), st_dev, sizeof(SlotState) * nslots, cudaMemcpyDeviceToHost, ctx->stream));
      HP_CUDA(cudaStreamSynchronize(ctx->stream));
      for (int sl : done) {
        SlotState& S = host[sl];
        const int L = S.lat;
        const int dof = pb.lats[L].op_kind == HP_OP_WILSON ? dof_wilson : pb.lats[L].parts;
        res.qj[L][(size_t)(S.m - pb.first[L]) * dof + S.a] = S.q;
        res.qb[L][(size_t)(S.m - pb.first[L]) * dof + S.a] = make_double2(S.gauss, S.gauss + S.radau * S.rnorm2);
        res.stats.rhs_solved += 1;
        res.stats.iterations_total += S.iters;
        res.stats.iterations_max = std::max(res.stats.iterations_max, S.iters);
        res.stats.iterations_min = std::min(res.stats.iterations_min, S.iters);
        res.stats.reliable_updates += S.updates;
        res.stats.sloppy_matvecs += S.sloppy_mv;
        res.stats.fp64_matvecs += S.fp64_mv;
        res.stats.group_updates += S.gupdates;
        double rel = S.bnorm2 > 0 ? std::sqrt(S.true_res2 / S.bnorm2) : 0.0;
        res.stats.max_true_residual = std::max(res.stats.max_true_residual, rel);
        if (S.status == SLOT_FAIL) {
          res.stats.n_unconverged += 1;
          res.unconverged = true;
        }
        S.status = SLOT_EMPTY;
      }
    }
  }
  if (gexec) cudaGraphExecDestroy(gexec);
  if (res.stats.rhs_solved == 0) res.stats.iterations_min = 0;
  res.stats.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return status;
}
