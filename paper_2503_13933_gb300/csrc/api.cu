#include <stdlib.h>
// C ABI: problem and factor objects, sweeps, greedy solve (Algorithm 1 with a growing
// mode count), residuals and grid reconstruction (Eq. 13).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "taps_internal.cuh"

int taps_weighted_ready(const taps_problem* P);
int taps_project_sources_dim(const taps_dim* d, const taps_source* sources, int Rf, int dimIndex, double* d_q,
                             cudaStream_t s);
int taps_project_source(const taps_dim* d, int kind, const double* par, const double* nodal_host,
                        double* d_q_free, cudaStream_t s);

int taps_sweep_setup(int dev, int num_sms, int* coop_blocks);

// ---------------------------------------------------------------------------------
// Profiling: launch counts always; CUDA events around launches when enabled.
// ---------------------------------------------------------------------------------
int prof_begin(taps_problem* P, int cls) {
  ProfState* S = P->prof;
  if (!S) return -1;
  S->launches[cls] += 1;
  // without timing events a captured graph gets no event-record nodes between its
  // kernels (they would add a dependency hop per class)
  if (!S->events) return -1;
  if (S->capturing && (S->npool < 2 || S->npending >= 512)) return -1;  // no allocation / sync while capturing
  if (S->npending >= 512) {
    cudaStreamSynchronize(P->stream);
    prof_drain(P);
  }
  if (S->npool < 2) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -1;
    S->pool[S->npool++] = a;
    S->pool[S->npool++] = b;
  }
  ProfPending& pp = S->pending[S->npending];
  pp.cls = cls;
  pp.b = S->pool[--S->npool];
  pp.a = S->pool[--S->npool];
  // inside a capture the record must become an event-record node of the graph
  if (S->capturing) cudaEventRecordWithFlags(pp.a, P->stream, cudaEventRecordExternal);
  else cudaEventRecord(pp.a, P->stream);
  return S->npending++;
}

void prof_end(taps_problem* P, int cls, int token, double flops, double bytes) {
  ProfState* S = P->prof;
  if (!S) return;
  S->flops[cls] += flops;
  S->bytes[cls] += bytes;
  if (token >= 0) {
    if (S->capturing) cudaEventRecordWithFlags(S->pending[token].b, P->stream, cudaEventRecordExternal);
    else cudaEventRecord(S->pending[token].b, P->stream);
  }
}

// Read back the elapsed times of all pending launches (the stream has been
// synchronised by the caller) and return the events to the pool.
void prof_drain(taps_problem* P) {
  ProfState* S = P->prof;
  if (!S) return;
  for (int i = 0; i < S->npending; ++i) {
    ProfPending& pp = S->pending[i];
    float ms = 0.f;
    if (cudaEventSynchronize(pp.b) == cudaSuccess && cudaEventElapsedTime(&ms, pp.a, pp.b) == cudaSuccess)
      S->ms[pp.cls] += ms;
    if (S->npool + 2 <= 1024) {
      S->pool[S->npool++] = pp.a;
      S->pool[S->npool++] = pp.b;
    } else {
      cudaEventDestroy(pp.a);
      cudaEventDestroy(pp.b);
    }
  }
  S->npending = 0;
}

// ---------------------------------------------------------------------------------
// Sweep graphs: one sweep plus one residual evaluation, captured once per
// (factors, M, precision, solver, residual kind, workspace) and replayed.
// ---------------------------------------------------------------------------------
struct SweepGraph {
  const taps_factors* U;
  int M, precision, solver, res_kind, ws_M;
  bool events;                   // captured with timing-event nodes
  bool failed;
  bool c0_skip;                  // its sweep reuses dim 0's coefficients from before the replay
  cudaGraph_t g;
  cudaGraphExec_t exec;
  long long dl[TAPS_PROF_NUM];   // per-replay profiling increments
  double dfl[TAPS_PROF_NUM], dby[TAPS_PROF_NUM];
  int nrec;
  ProfPending recs[512];         // events recorded by the graph's own event nodes
};

static void graph_destroy(taps_problem* P) {
  SweepGraph* G = (SweepGraph*)P->graph;
  if (!G) return;
  if (G->exec) cudaGraphExecDestroy(G->exec);
  if (G->g) cudaGraphDestroy(G->g);
  for (int i = 0; i < G->nrec; ++i) {
    cudaEventDestroy(G->recs[i].a);
    cudaEventDestroy(G->recs[i].b);
  }
  delete G;
  P->graph = nullptr;
}

static int graph_build(taps_problem* P, taps_factors* U, int prec, int solver, int res_kind) {
  graph_destroy(P);
  SweepGraph* G = new SweepGraph();
  memset((void*)G, 0, sizeof(SweepGraph));
  G->U = U;
  G->M = U->M;
  G->precision = prec;
  G->solver = solver;
  G->res_kind = res_kind;
  G->ws_M = P->ws_M;
  G->events = P->prof->events;
  P->graph = G;
  ProfState* S = P->prof;
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  prof_drain(P);
  long long l0[TAPS_PROF_NUM];
  double f0[TAPS_PROF_NUM], b0[TAPS_PROF_NUM];
  for (int c = 0; c < TAPS_PROF_NUM; ++c) { l0[c] = S->launches[c]; f0[c] = S->flops[c]; b0[c] = S->bytes[c]; }
  while (S->npool < 512) {   // events for the graph's event nodes, created before capture
    cudaEvent_t ev;
    if (cudaEventCreate(&ev) != cudaSuccess) break;
    S->pool[S->npool++] = ev;
  }
  cudaStream_t saved = P->stream;
  P->stream = P->cap_stream;
  int st = TAPS_OK;
  S->capturing = true;
  // capture runs nothing: the coefficient state is the pre-capture one until a replay
  const int c0_before = P->c0_valid, c0_M_before = P->c0_M;
  P->c0_skipped = 0;
  if (cudaStreamBeginCapture(P->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    st = TAPS_ERR_CUDA;
  } else {
    st = taps_sweep_enqueue(P, U, prec, solver, 1, 0);
    if (st == TAPS_OK) st = taps_residual_enqueue(P, U, res_kind, !taps_low_prec(prec), 0);
    if (st == TAPS_OK) st = taps_results_to_host(P, 2 * U->M * P->D, taps_residual_npart(P, res_kind));
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(P->cap_stream, &g);
    if (ce != cudaSuccess || g == nullptr) st = (st == TAPS_OK) ? TAPS_ERR_CUDA : st;
    G->g = g;
  }
  G->c0_skip = P->c0_skipped != 0;
  P->c0_valid = c0_before;
  P->c0_M = c0_M_before;
  P->stream = saved;
  S->capturing = false;
  cudaGetLastError();
  for (int c = 0; c < TAPS_PROF_NUM; ++c) {
    G->dl[c] = S->launches[c] - l0[c];
    G->dfl[c] = S->flops[c] - f0[c];
    G->dby[c] = S->bytes[c] - b0[c];
    S->launches[c] = l0[c];
    S->flops[c] = f0[c];
    S->bytes[c] = b0[c];
  }
  for (int i = 0; i < S->npending; ++i) G->recs[G->nrec++] = S->pending[i];
  S->npending = 0;
  if (st == TAPS_OK && cudaGraphInstantiate(&G->exec, G->g, 0) != cudaSuccess) {
    cudaGetLastError();
    st = TAPS_ERR_CUDA;
  }
  if (st != TAPS_OK) G->failed = true;
  return st;
}

// ---------------------------------------------------------------------------------
// Device-side solve loop: one CUDA graph whose conditional WHILE node repeats
// {sweep, Eq. 42 residual, decision} without returning to the host.  The decision
// kernel forms the factor change and rho_42 from the device partial sums in the order
// the host's finish functions use (so the stopping sweep and the factors are those of
// the host loop), records them and sets the loop condition.
// ---------------------------------------------------------------------------------
struct LoopRanges {
  int cta0[TAPS_MAX_DIMS + 1];
};

__global__ void solve_decide_kernel(cudaGraphConditionalHandle h, const double* __restrict__ scal, int M, int D,
                                    const double* __restrict__ part, LoopRanges rg, double res_tol,
                                    double als_tol, int max_sweeps, int* __restrict__ state,
                                    double* __restrict__ hist, int cap, const int* __restrict__ status) {
  if (threadIdx.x != 0) return;
  double change = 0.0;
  for (int d = 0; d < D; ++d) {
    double dif = 0.0, n2 = 0.0;
    for (int m = 0; m < M; ++m) {
      dif += scal[(size_t)d * 2 * M + 2 * m];
      n2 += scal[(size_t)d * 2 * M + 2 * m + 1];
    }
    change = fmax(change, n2 > 0.0 ? sqrt(dif / n2) : INFINITY);
  }
  double rho = 0.0;
  for (int d = 0; d < D; ++d) {
    double r2 = 0.0, f2 = 0.0;
    for (int b = rg.cta0[d]; b < rg.cta0[d + 1]; ++b) {
      r2 += part[2 * b];
      f2 += part[2 * b + 1];
    }
    rho = fmax(rho, f2 > 0.0 ? sqrt(r2 / f2) : INFINITY);
  }
  const int it = state[0];
  if (it < cap) {
    hist[2 * it] = rho;
    hist[2 * it + 1] = change;
  }
  state[0] = it + 1;
  const int st = *status;
  const bool finite = isfinite(rho) && isfinite(change);
  state[1] = st;
  state[2] = finite ? 1 : 0;
  const bool more = st == 0 && finite && !(rho <= res_tol) && !(change <= als_tol) && it + 1 < max_sweeps;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

struct LoopGraph {
  const taps_factors* U;
  int M, precision, solver, ws_M, max_sweeps;
  double res_tol, als_tol;
  bool failed;
  bool c0_skip;       // the body's sweep reuses dim 0's coefficients (see SweepGraph)
  cudaGraph_t g;
  cudaGraphExec_t exec;
  cudaGraphConditionalHandle h;
  int* d_state;       // [iterations, status, finite]
  double* d_hist;     // [max_sweeps][rho, change]
  int* h_state;       // pinned mirrors
  double* h_hist;
  long long dl[TAPS_PROF_NUM];   // per-iteration profiling increments
  double dfl[TAPS_PROF_NUM], dby[TAPS_PROF_NUM];
};

static void loop_destroy(taps_problem* P) {
  LoopGraph* L = (LoopGraph*)P->loop_graph;
  if (!L) return;
  if (L->exec) cudaGraphExecDestroy(L->exec);
  if (L->g) cudaGraphDestroy(L->g);
  cudaFree(L->d_state);
  cudaFree(L->d_hist);
  if (L->h_state) cudaFreeHost(L->h_state);
  if (L->h_hist) cudaFreeHost(L->h_hist);
  delete L;
  P->loop_graph = nullptr;
}

static int loop_build(taps_problem* P, taps_factors* U, int prec, int solver, double res_tol, double als_tol,
                      int max_sweeps) {
  loop_destroy(P);
  LoopGraph* L = new LoopGraph();
  memset((void*)L, 0, sizeof(LoopGraph));
  L->U = U;
  L->M = U->M;
  L->precision = prec;
  L->solver = solver;
  L->ws_M = P->ws_M;
  L->max_sweeps = max_sweeps;
  L->res_tol = res_tol;
  L->als_tol = als_tol;
  P->loop_graph = L;
  int st = TAPS_OK;
  do {
    if ((st = taps_alloc((void**)&L->d_state, sizeof(int) * 4)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&L->d_hist, sizeof(double) * 2 * (size_t)max_sweeps)) != TAPS_OK) break;
    if (cudaMallocHost((void**)&L->h_state, sizeof(int) * 4) != cudaSuccess ||
        cudaMallocHost((void**)&L->h_hist, sizeof(double) * 2 * (size_t)max_sweeps) != cudaSuccess) {
      st = TAPS_ERR_OOM;
      break;
    }
    if (cudaGraphCreate(&L->g, 0) != cudaSuccess ||
        cudaGraphConditionalHandleCreate(&L->h, L->g, 1, cudaGraphCondAssignDefault) != cudaSuccess) {
      st = TAPS_ERR_CUDA;
      break;
    }
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = L->h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t node;
    if (cudaGraphAddNode(&node, L->g, nullptr, nullptr, 0, &cp) != cudaSuccess) {
      st = TAPS_ERR_CUDA;
      break;
    }
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    LoopRanges rg;
    memset(&rg, 0, sizeof(rg));
    taps_als_partial_ranges(P, rg.cta0);
    ProfState* S = P->prof;
    long long l0[TAPS_PROF_NUM];
    double f0[TAPS_PROF_NUM], b0[TAPS_PROF_NUM];
    for (int c = 0; c < TAPS_PROF_NUM; ++c) { l0[c] = S->launches[c]; f0[c] = S->flops[c]; b0[c] = S->bytes[c]; }
    cudaStream_t saved = P->stream;
    P->stream = P->cap_stream;
    S->capturing = true;
    const int c0_before = P->c0_valid, c0_M_before = P->c0_M;
    P->c0_skipped = 0;
    if (cudaStreamBeginCaptureToGraph(P->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) !=
        cudaSuccess) {
      st = TAPS_ERR_CUDA;
    } else {
      st = taps_sweep_enqueue(P, U, prec, solver, 1, 0);
      if (st == TAPS_OK) st = taps_residual_enqueue(P, U, TAPS_RES_ALS, !taps_low_prec(prec), 0);
      if (st == TAPS_OK) {
        solve_decide_kernel<<<1, 32, 0, P->stream>>>(L->h, P->d_scal, U->M, P->D, P->d_partial, rg, res_tol, als_tol,
                                                     max_sweeps, L->d_state, L->d_hist, max_sweeps, P->d_status);
        if (cudaGetLastError() != cudaSuccess) st = TAPS_ERR_CUDA;
      }
      cudaGraph_t out = nullptr;
      if (cudaStreamEndCapture(P->cap_stream, &out) != cudaSuccess) st = (st == TAPS_OK) ? TAPS_ERR_CUDA : st;
    }
    L->c0_skip = P->c0_skipped != 0;
    P->c0_valid = c0_before;
    P->c0_M = c0_M_before;
    P->stream = saved;
    S->capturing = false;
    cudaGetLastError();
    for (int c = 0; c < TAPS_PROF_NUM; ++c) {
      L->dl[c] = S->launches[c] - l0[c];
      L->dfl[c] = S->flops[c] - f0[c];
      L->dby[c] = S->bytes[c] - b0[c];
      S->launches[c] = l0[c];
      S->flops[c] = f0[c];
      S->bytes[c] = b0[c];
    }
    S->npending = 0;
    if (st == TAPS_OK && cudaGraphInstantiate(&L->exec, L->g, 0) != cudaSuccess) {
      cudaGetLastError();
      st = TAPS_ERR_CUDA;
    }
  } while (0);
  if (st != TAPS_OK) L->failed = true;
  return st;
}

// Runs up to max_sweeps sweeps on the device.  Returns TAPS_ERR_CUDA with *fallback = 1
// when the loop graph is unavailable (the caller runs the host loop).  On return,
// *done sweeps ran, hist_rho / hist_change (device order) hold their values.
static int loop_solve(taps_problem* P, taps_factors* U, int prec, int solver, double res_tol, double als_tol,
                      int max_sweeps, int* done, const double** hist, int* fallback) {
  *fallback = 0;
  *done = 0;
  LoopGraph* L = (LoopGraph*)P->loop_graph;
  bool match = L && L->U == U && L->M == U->M && L->precision == prec && L->solver == solver &&
               L->ws_M == P->ws_M && L->max_sweeps == max_sweeps && L->res_tol == res_tol &&
               L->als_tol == als_tol;
  if (match && L->failed) {
    *fallback = 1;
    return TAPS_ERR_CUDA;
  }
  if (!match) {
    if (taps_lu_needs_tuning(P, solver, U->M)) {   // the block-elimination tuner runs eagerly
      *fallback = 1;
      return TAPS_ERR_CUDA;
    }
    TAPS_TRY(taps_fd_prepare_all(P, solver, U->M));
    if (loop_build(P, U, prec, solver, res_tol, als_tol, max_sweeps) != TAPS_OK) {
      *fallback = 1;
      return TAPS_ERR_CUDA;
    }
    L = (LoopGraph*)P->loop_graph;
  }
  cudaStream_t s = P->stream;
  if (L->c0_skip && !(P->c0_valid && P->c0_M == U->M)) TAPS_TRY(taps_coefficients(P, 0, U->M));
  TAPS_CUDA(cudaMemsetAsync(L->d_state, 0, sizeof(int) * 4, s));
  TAPS_CUDA(cudaGraphLaunch(L->exec, s));
  P->c0_valid = 1;   // every body ends with the last dim's refresh forming them
  P->c0_M = U->M;
  TAPS_CUDA(cudaMemcpyAsync(L->h_state, L->d_state, sizeof(int) * 4, cudaMemcpyDeviceToHost, s));
  TAPS_CUDA(cudaMemcpyAsync(L->h_hist, L->d_hist, sizeof(double) * 2 * (size_t)max_sweeps, cudaMemcpyDeviceToHost,
                            s));
  TAPS_CUDA(cudaStreamSynchronize(s));
  const int n = std::min(L->h_state[0], max_sweeps);
  ProfState* S = P->prof;
  for (int c = 0; c < TAPS_PROF_NUM; ++c) {
    S->launches[c] += L->dl[c] * n;
    S->flops[c] += L->dfl[c] * n;
    S->bytes[c] += L->dby[c] * n;
  }
  *done = n;
  *hist = L->h_hist;
  if (L->h_state[1] != TAPS_DEV_OK) {
    const int dev = L->h_state[1];
    TAPS_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), s));
    TAPS_CUDA(cudaStreamSynchronize(s));
    return taps_status_from_device(dev);
  }
  if (!L->h_state[2]) return TAPS_ERR_NONFINITE;
  return TAPS_OK;
}

// One sweep + residual through the cached graph (built on first use).  Returns
// TAPS_ERR_CUDA with *fallback = 1 if capture is unavailable (caller runs eagerly).
static int graph_sweep(taps_problem* P, taps_factors* U, int prec, int solver, int res_kind,
                       double* change, double* rho, int* fallback) {
  *fallback = 0;
  SweepGraph* G = (SweepGraph*)P->graph;
  bool match = G && G->U == U && G->M == U->M && G->precision == prec && G->solver == solver &&
               G->res_kind == res_kind && G->ws_M == P->ws_M && G->events == P->prof->events;
  if (match && G->failed) {
    *fallback = 1;
    return TAPS_ERR_CUDA;
  }
  if (!match && taps_lu_needs_tuning(P, solver, U->M)) {
    *fallback = 1;   // run this sweep directly: the block-elimination tuner needs it
    return TAPS_ERR_CUDA;
  }
  if (!match) {
    TAPS_TRY(taps_fd_prepare_all(P, solver, U->M));
    if (graph_build(P, U, prec, solver, res_kind) != TAPS_OK) {
      *fallback = 1;
      return TAPS_ERR_CUDA;
    }
    G = (SweepGraph*)P->graph;
  }
  if (G->c0_skip && !(P->c0_valid && P->c0_M == U->M)) TAPS_TRY(taps_coefficients(P, 0, U->M));
  TAPS_CUDA(cudaGraphLaunch(G->exec, P->stream));
  P->c0_valid = 1;   // the sweep's last dim formed them
  P->c0_M = U->M;
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  ProfState* S = P->prof;
  for (int c = 0; c < TAPS_PROF_NUM; ++c) {
    S->launches[c] += G->dl[c];
    S->flops[c] += G->dfl[c];
    S->bytes[c] += G->dby[c];
  }
  if (S->events)
    for (int i = 0; i < G->nrec; ++i) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, G->recs[i].a, G->recs[i].b) == cudaSuccess) S->ms[G->recs[i].cls] += ms;
    }
  cudaGetLastError();
  TAPS_TRY(taps_sweep_finish(P, U, change));
  return taps_residual_finish(P, U, res_kind, rho);
}

extern "C" int taps_profile_reset(taps_problem* P, int enable_events) {
  if (!P || !P->prof) return TAPS_ERR_INVALID_ARG;
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  prof_drain(P);
  ProfState* S = P->prof;
  for (int c = 0; c < TAPS_PROF_NUM; ++c) {
    S->launches[c] = 0;
    S->ms[c] = S->flops[c] = S->bytes[c] = 0.0;
  }
  S->events = enable_events != 0;
  return TAPS_OK;
}

extern "C" int taps_profile_get(taps_problem* P, int cls, long long* launches, double* ms,
                                double* flops, double* bytes) {
  if (!P || !P->prof || cls < 0 || cls >= TAPS_PROF_NUM) return TAPS_ERR_INVALID_ARG;
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  prof_drain(P);
  ProfState* S = P->prof;
  if (launches) *launches = S->launches[cls];
  if (ms) *ms = S->ms[cls];
  if (flops) *flops = S->flops[cls];
  if (bytes) *bytes = S->bytes[cls];
  return TAPS_OK;
}

// ---------------------------------------------------------------------------------
// Problem
// ---------------------------------------------------------------------------------
static void free_ws(taps_problem* P) {
  for (int d = 0; d < TAPS_MAX_DIMS; ++d) {
    cudaFree(P->d_gram[d]);
    cudaFree(P->d_h[d]);
    P->d_gram[d] = P->d_h[d] = nullptr;
  }
  for (int d = 0; d < TAPS_MAX_DIMS; ++d) {
    cudaFree(P->d_Usnap[d]);
    P->d_Usnap[d] = nullptr;
  }
  loop_destroy(P);
  cudaFree(P->d_C);
  cudaFree(P->d_c);
  cudaFree(P->d_Call);
  cudaFree(P->d_call);
  cudaFree(P->d_ticket);
  P->d_Call = P->d_call = nullptr;
  P->d_ticket = nullptr;
  cudaFree(P->d_F);
  cudaFree(P->d_blocks);
  cudaFree(P->d_lu);
  cudaFree(P->d_Y);
  cudaFree(P->d_Uold);
  cudaFree(P->d_md);
  P->d_md = nullptr;
  cudaFree(P->d_fdw);
  P->d_fdw = nullptr;
  cudaFree(P->d_partial);
  cudaFree(P->d_scal);
  cudaFree(P->d_bigG);
  cudaFree(P->d_Yres);
  P->d_Yres = nullptr;
  cudaFree(P->d_ticket_all);
  P->d_ticket_all = nullptr;
  if (P->h_scal) cudaFreeHost(P->h_scal);
  if (P->h_part) cudaFreeHost(P->h_part);
  P->h_part = nullptr;
  graph_destroy(P);
  P->d_C = P->d_c = P->d_F = P->d_blocks = P->d_lu = P->d_Y = P->d_Uold = nullptr;
  P->d_partial = P->d_scal = P->d_bigG = P->h_scal = nullptr;
  P->ws_M = 0;
}

extern "C" void taps_problem_destroy(taps_problem* P) {
  if (!P) return;
  if (P->stream) cudaStreamSynchronize(P->stream);
  free_ws(P);
  for (int d = 0; d < TAPS_MAX_DIMS; ++d) {
    cudaFree(P->d_q[d]);
    cudaFree(P->d_pq[d]);
    cudaFree(P->d_opband[d]);
  }
  cudaFree(P->d_status);
  cudaFree(P->d_bar);
  cudaFree(P->d_beta);
  cudaFree(P->d_evalbuf);
  cudaFree(P->d_wbuf);
  if (P->h_status) cudaFreeHost(P->h_status);
  if (P->cap_stream) cudaStreamDestroy(P->cap_stream);
  if (P->prof) {
    for (int i = 0; i < P->prof->npending; ++i) {
      cudaEventDestroy(P->prof->pending[i].a);
      cudaEventDestroy(P->prof->pending[i].b);
    }
    for (int i = 0; i < P->prof->npool; ++i) cudaEventDestroy(P->prof->pool[i]);
    delete P->prof;
  }
  delete P;
}

int taps_ws_ensure(taps_problem* P, int M) {
  if (M <= P->ws_M) return TAPS_OK;
  if (P->stream) TAPS_CUDA(cudaStreamSynchronize(P->stream));
  free_ws(P);
  P->c0_valid = 0;
  int nbmax = 0, D = P->D;
  size_t part = 0, bigG = 0, yres = 0, part_all = 0;
  for (int d = 0; d < D; ++d) {
    const taps_dim* dm = P->dims[d];
    int nops = P->tt.nops[d];
    nbmax = std::max(nbmax, dm->nb);
    TAPS_TRY(taps_alloc((void**)&P->d_gram[d], sizeof(double) * nops * M * M));
    TAPS_TRY(taps_alloc((void**)&P->d_h[d], sizeof(double) * P->Rf * M));
    TAPS_TRY(taps_alloc((void**)&P->d_Usnap[d], sizeof(double) * dm->nf * M));
    size_t gp = (size_t)((dm->nf + 7) / 8) * (nops * M * M + P->Rf * M);
    part = std::max(part, gp);
    part_all += gp;
    size_t NC = (size_t)nops * M + P->Rf;
    bigG += NC * NC;
    yres += (size_t)nops * dm->nf * M;
  }
  size_t als_part = 0;
  for (int d = 0; d < D; ++d) als_part += 2 * (((size_t)P->dims[d]->nf + 7) / 8);   // 8 rows per CTA
  part = std::max(part, als_part);
  // the all-dims Gram refresh needs every dim's chunk partials at once: allowed up to 32 MB
  P->gram_all_ok = part_all <= ((size_t)1 << 22);
  if (P->gram_all_ok) part = std::max(part, part_all);
  part = std::max(part, (size_t)3 * 64);
  size_t MM = (size_t)M * M;
  int nfm = P->nf_max;
  const size_t cs = (size_t)P->tt.cs;   // TAPS_NUM_OPS unless weighted operators add slots
  TAPS_TRY(taps_alloc((void**)&P->d_C, sizeof(double) * cs * MM));
  TAPS_TRY(taps_alloc((void**)&P->d_c, sizeof(double) * P->Rf * M));
  TAPS_TRY(taps_alloc((void**)&P->d_Call, sizeof(double) * D * cs * MM));
  TAPS_TRY(taps_alloc((void**)&P->d_call, sizeof(double) * D * P->Rf * M));
  TAPS_TRY(taps_alloc((void**)&P->d_ticket, sizeof(unsigned) * 64));   // >= M / 8 + 1
  TAPS_CUDA(cudaMemsetAsync(P->d_ticket, 0, sizeof(unsigned) * 64, P->stream));
  TAPS_TRY(taps_alloc((void**)&P->d_ticket_all, sizeof(unsigned) * 32 * TAPS_MAX_DIMS));
  TAPS_CUDA(cudaMemsetAsync(P->d_ticket_all, 0, sizeof(unsigned) * 32 * TAPS_MAX_DIMS, P->stream));
  TAPS_TRY(taps_alloc((void**)&P->d_F, sizeof(double) * nfm * M));
  TAPS_TRY(taps_alloc((void**)&P->d_blocks, sizeof(double) * nfm * nbmax * MM));
  TAPS_TRY(taps_alloc((void**)&P->d_lu, sizeof(double) * MM));
  TAPS_TRY(taps_alloc((void**)&P->d_Y, sizeof(double) * cs * nfm * M));
  TAPS_TRY(taps_alloc((void**)&P->d_Uold, sizeof(double) * nfm * M));
  TAPS_TRY(taps_alloc((void**)&P->d_fdw, sizeof(double) * taps_fdw_scratch_doubles(nfm, M)));
  TAPS_TRY(taps_alloc((void**)&P->d_md, sizeof(double) * taps_md_scratch_doubles(nfm, M, P->Rf)));
  TAPS_CUDA(cudaMemsetAsync(P->d_md, 0, sizeof(double) * taps_md_scratch_doubles(nfm, M, P->Rf), P->stream));
  TAPS_TRY(taps_alloc((void**)&P->d_partial, sizeof(double) * part));
  TAPS_TRY(taps_alloc((void**)&P->d_scal, sizeof(double) * 2 * M * D + 64));
  TAPS_TRY(taps_alloc((void**)&P->d_bigG, sizeof(double) * bigG));
  TAPS_TRY(taps_alloc((void**)&P->d_Yres, sizeof(double) * yres));
  TAPS_CUDA(cudaMallocHost((void**)&P->h_scal, sizeof(double) * (2 * M * D + 64)));
  TAPS_CUDA(cudaMallocHost((void**)&P->h_part, sizeof(double) * part));
  P->partial_len = part;
  P->bigG_len = bigG;
  P->ws_M = M;
  return TAPS_OK;
}

extern "C" int taps_problem_create(taps_dim* const* dims, int D, const taps_term* terms, int R,
                                   const taps_source* sources, int Rf, void* stream,
                                   taps_problem** out) {
  if (!out) return TAPS_ERR_INVALID_ARG;
  *out = nullptr;
  if (!dims || !terms || !sources || D < 1 || D > TAPS_MAX_DIMS || R < 1 || R > TAPS_MAX_TERMS ||
      Rf < 1 || Rf > TAPS_MAX_SOURCES)
    return TAPS_ERR_INVALID_ARG;
  for (int d = 0; d < D; ++d)
    if (!dims[d]) return TAPS_ERR_INVALID_ARG;
  for (int t = 0; t < R; ++t)
    for (int d = 0; d < D; ++d) {
      const int op = terms[t].op[d];
      const bool plain = op >= 0 && op < TAPS_NUM_OPS;
      const bool weighted = op >= TAPS_OP_WEIGHTED && op < TAPS_OP_WEIGHTED + TAPS_MAX_WEIGHTED;
      if (!plain && !weighted) return TAPS_ERR_INVALID_ARG;
    }
  for (int d = 0; d < D; ++d) {   // distinct operators per dim
    int distinct = 0;
    for (int t = 0; t < R; ++t) {
      bool seen = false;
      for (int u = 0; u < t; ++u) seen = seen || terms[u].op[d] == terms[t].op[d];
      distinct += seen ? 0 : 1;
    }
    if (distinct > TAPS_MAX_SLOTS) return TAPS_ERR_INVALID_ARG;
  }
  for (int r = 0; r < Rf; ++r)
    for (int d = 0; d < D; ++d) {
      int k = sources[r].kind[d];
      if (k < TAPS_SRC_CONST || k > TAPS_SRC_OPVEC_FULL) return TAPS_ERR_INVALID_ARG;
      if ((k == TAPS_SRC_NODAL || k == TAPS_SRC_OPVEC || k == TAPS_SRC_OPVEC_FULL) && !sources[r].nodal[d])
        return TAPS_ERR_INVALID_ARG;
      if ((k == TAPS_SRC_OPVEC || k == TAPS_SRC_OPVEC_FULL) &&
          (sources[r].par[d][0] < 0 || sources[r].par[d][0] >= TAPS_NUM_OPS))
        return TAPS_ERR_INVALID_ARG;
    }
  taps_problem* P = new taps_problem();
  memset((void*)P, 0, sizeof(taps_problem));
  P->D = D;
  P->R = R;
  P->Rf = Rf;
  P->stream = (cudaStream_t)stream;
  P->prof = new ProfState();
  memset((void*)P->prof, 0, sizeof(ProfState));
  P->tt.D = D;
  P->tt.R = R;
  P->tt.Rf = Rf;
  // Distinct operator slots per dim, in order of first appearance in the terms.
  for (int d = 0; d < D; ++d) {
    P->dims[d] = dims[d];
    P->nf_max = std::max(P->nf_max, dims[d]->nf);
    int n = 0;
    for (int t = 0; t < R; ++t) {
      int op = terms[t].op[d], slot = -1;
      for (int j = 0; j < n; ++j)
        if (P->ops[d][j] == op) slot = j;
      if (slot < 0) {
        slot = n;
        P->ops[d][n++] = op;
      }
      P->tt.oi[t][d] = (signed char)slot;
      if (op >= TAPS_OP_WEIGHTED) {
        P->has_weighted = true;
        P->wuse[d] |= 1ull << (op - TAPS_OP_WEIGHTED);
      }
    }
    P->tt.nops[d] = n;
    P->tt.cs = std::max(P->tt.cs, n);
  }
  P->tt.cs = std::max(P->tt.cs, TAPS_NUM_OPS);
  for (int t = 0; t < R; ++t) P->tt.alpha[t] = terms[t].alpha;
  std::vector<double> hbeta(Rf);
  for (int r = 0; r < Rf; ++r) hbeta[r] = sources[r].beta;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&P->num_sms, cudaDevAttrMultiProcessorCount, dev);
  int st = TAPS_OK;
  do {
    if ((st = taps_alloc((void**)&P->d_status, sizeof(int))) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&P->d_bar, 2 * sizeof(unsigned))) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&P->d_beta, sizeof(double) * Rf)) != TAPS_OK) break;
    if (cudaMemcpy(P->d_beta, hbeta.data(), sizeof(double) * Rf, cudaMemcpyHostToDevice) != cudaSuccess) {
      st = TAPS_ERR_CUDA;
      break;
    }
    P->tt.beta = P->d_beta;
    if (cudaMallocHost((void**)&P->h_status, sizeof(int)) != cudaSuccess) { st = TAPS_ERR_OOM; break; }
    *P->h_status = 0;
    if (cudaStreamCreateWithFlags(&P->cap_stream, cudaStreamNonBlocking) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    if (cudaMemsetAsync(P->d_status, 0, sizeof(int), P->stream) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    for (int d = 0; d < D && st == TAPS_OK; ++d) {
      const taps_dim* dm = dims[d];
      int nops = P->tt.nops[d];
      size_t bandsz = (size_t)dm->nf * dm->nb;
      if ((st = taps_alloc((void**)&P->d_opband[d], sizeof(double) * nops * bandsz)) != TAPS_OK) break;
      for (int j = 0; j < nops; ++j) {
        cudaError_t ce = P->ops[d][j] < TAPS_NUM_OPS
                             ? cudaMemcpyAsync(P->d_opband[d] + j * bandsz, dm->d_band + (size_t)P->ops[d][j] * bandsz,
                                               sizeof(double) * bandsz, cudaMemcpyDeviceToDevice, P->stream)
                             : cudaMemsetAsync(P->d_opband[d] + j * bandsz, 0, sizeof(double) * bandsz, P->stream);
        if (ce != cudaSuccess) st = TAPS_ERR_CUDA;
      }
      if (st != TAPS_OK) break;
      if ((st = taps_alloc((void**)&P->d_q[d], sizeof(double) * Rf * dm->nf)) != TAPS_OK) break;
      st = taps_project_sources_dim(dm, sources, Rf, d, P->d_q[d], P->stream);
    }
    if (st != TAPS_OK) break;
    if ((st = taps_sweep_setup(dev, P->num_sms, &P->coop_blocks)) != TAPS_OK) break;
    st = taps_check_status(P->d_status, P->stream);
  } while (0);
  if (st != TAPS_OK) {
    taps_problem_destroy(P);
    return st;
  }
  *out = P;
  return TAPS_OK;
}

int taps_dim_weighted_bands(const taps_dim* d, int count, const int* base, const int* slot, const double* d_w,
                            double* bands, cudaStream_t stream);

extern "C" int taps_problem_set_weighted_ops(taps_problem* P, int d, int count, const int* base,
                                             const double* weights) {
  if (!P || !base || !weights || d < 0 || d >= P->D || count < 1 || count > TAPS_MAX_WEIGHTED)
    return TAPS_ERR_INVALID_ARG;
  for (int j = 0; j < count; ++j)
    if (base[j] != TAPS_OP_K && base[j] != TAPS_OP_M && base[j] != TAPS_OP_G) return TAPS_ERR_INVALID_ARG;
  const taps_dim* dm = P->dims[d];
  const size_t n = (size_t)dm->n, need = (size_t)count * n;
  if (need > P->wbuf_cap) {
    if (P->stream) TAPS_CUDA(cudaStreamSynchronize(P->stream));
    cudaFree(P->d_wbuf);
    P->d_wbuf = nullptr;
    P->wbuf_cap = 0;
    TAPS_TRY(taps_alloc((void**)&P->d_wbuf, sizeof(double) * need));
    P->wbuf_cap = need;
  }
  TAPS_CUDA(cudaMemcpyAsync(P->d_wbuf, weights, sizeof(double) * need, cudaMemcpyHostToDevice, P->stream));
  int slot[TAPS_MAX_WEIGHTED];
  for (int j = 0; j < count; ++j) slot[j] = -1;
  for (int s = 0; s < P->tt.nops[d]; ++s) {
    const int j = P->ops[d][s] - TAPS_OP_WEIGHTED;
    if (j >= 0 && j < count) slot[j] = s;
  }
  TAPS_TRY(taps_dim_weighted_bands(dm, count, base, slot, P->d_wbuf, P->d_opband[d], P->stream));
  P->wdef[d] |= (count >= 64) ? ~0ull : ((1ull << count) - 1ull);
  // the staging buffer is reused by the next call: the copies above must be done
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return TAPS_OK;
}

// Every weighted operator the terms use has been defined.
int taps_weighted_ready(const taps_problem* P) {
  for (int d = 0; d < P->D; ++d)
    if (P->wuse[d] & ~P->wdef[d]) return TAPS_ERR_INVALID_ARG;
  return TAPS_OK;
}

extern "C" int taps_problem_copy_op(const taps_problem* P, int d, int op, double* host_out) {
  if (!P || !host_out || d < 0 || d >= P->D) return TAPS_ERR_INVALID_ARG;
  int slot = -1;
  for (int s = 0; s < P->tt.nops[d]; ++s)
    if (P->ops[d][s] == op) slot = s;
  if (slot < 0) return TAPS_ERR_INVALID_ARG;
  const size_t bandsz = (size_t)P->dims[d]->nf * P->dims[d]->nb;
  TAPS_CUDA(cudaMemcpyAsync(host_out, P->d_opband[d] + slot * bandsz, sizeof(double) * bandsz,
                            cudaMemcpyDeviceToHost, P->stream));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return TAPS_OK;
}

extern "C" int taps_problem_copy_source(const taps_problem* P, int r, int d, double* host_out) {
  if (!P || !host_out || r < 0 || r >= P->Rf || d < 0 || d >= P->D) return TAPS_ERR_INVALID_ARG;
  int nf = P->dims[d]->nf;
  TAPS_CUDA(cudaMemcpyAsync(host_out, P->d_q[d] + (size_t)r * nf, sizeof(double) * nf,
                            cudaMemcpyDeviceToHost, P->stream));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return TAPS_OK;
}

// ---------------------------------------------------------------------------------
// Factors
// ---------------------------------------------------------------------------------
extern "C" void taps_factors_destroy(taps_factors* U) {
  if (!U) return;
  for (int d = 0; d < TAPS_MAX_DIMS; ++d) cudaFree(U->d_U[d]);
  delete U;
}

extern "C" int taps_factors_create(const taps_problem* P, int M_cap, taps_factors** out) {
  if (!P || !out || M_cap < 1 || M_cap > TAPS_MAX_M) return TAPS_ERR_INVALID_ARG;
  taps_factors* U = new taps_factors();
  memset((void*)U, 0, sizeof(taps_factors));
  U->prob = P;
  U->M_cap = M_cap;
  for (int d = 0; d < P->D; ++d) {
    int st = taps_alloc((void**)&U->d_U[d], sizeof(double) * P->dims[d]->nf * M_cap);
    if (st != TAPS_OK) {
      taps_factors_destroy(U);
      return st;
    }
    cudaMemsetAsync(U->d_U[d], 0, sizeof(double) * P->dims[d]->nf * M_cap, P->stream);
  }
  *out = U;
  return TAPS_OK;
}

extern "C" int taps_factors_set(taps_factors* U, int M, const double* const* host_U) {
  if (!U || M < 0 || M > U->M_cap || (M > 0 && !host_U)) return TAPS_ERR_INVALID_ARG;
  const taps_problem* P = U->prob;
  for (int d = 0; d < P->D && M > 0; ++d) {
    if (!host_U[d]) return TAPS_ERR_INVALID_ARG;
    TAPS_CUDA(cudaMemcpyAsync(U->d_U[d], host_U[d], sizeof(double) * P->dims[d]->nf * M,
                              cudaMemcpyHostToDevice, P->stream));
  }
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  U->M = M;
  return TAPS_OK;
}

extern "C" int taps_factors_get(const taps_factors* U, double* const* host_U) {
  if (!U || !host_U) return TAPS_ERR_INVALID_ARG;
  const taps_problem* P = U->prob;
  for (int d = 0; d < P->D && U->M > 0; ++d) {
    if (!host_U[d]) return TAPS_ERR_INVALID_ARG;
    TAPS_CUDA(cudaMemcpyAsync(host_U[d], U->d_U[d], sizeof(double) * P->dims[d]->nf * U->M,
                              cudaMemcpyDeviceToHost, P->stream));
  }
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return TAPS_OK;
}

extern "C" int taps_factors_M(const taps_factors* U) { return U ? U->M : -1; }

extern "C" int taps_factors_copy(taps_factors* dst, const taps_factors* src) {
  if (!dst || !src || dst->prob != src->prob || src->M > dst->M_cap) return TAPS_ERR_INVALID_ARG;
  const taps_problem* P = src->prob;
  for (int d = 0; d < P->D && src->M > 0; ++d)
    TAPS_CUDA(cudaMemcpyAsync(dst->d_U[d], src->d_U[d], sizeof(double) * P->dims[d]->nf * src->M,
                              cudaMemcpyDeviceToDevice, P->stream));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  dst->M = src->M;
  return TAPS_OK;
}

// Gram matrix of the 3 Mx columns [A | B | A - B] of one dim (A and B padded with zero
// columns to Mx = max(MA, MB)); one CTA per entry.  The difference columns are formed
// here, exactly as the telescoped change below needs them.
__device__ __forceinline__ double pair_col(const double* UA, const double* UB, int MA, int MB, int Mx,
                                           int nf, int c, int i) {
  const int blk = c / Mx, m = c % Mx;
  const double a = m < MA ? UA[(size_t)m * nf + i] : 0.0;
  const double b = m < MB ? UB[(size_t)m * nf + i] : 0.0;
  return blk == 0 ? a : (blk == 1 ? b : a - b);
}

__global__ void pair_gram_kernel(const double* __restrict__ UA, const double* __restrict__ UB, int nf, int MA,
                                 int MB, int Mx, double* __restrict__ G) {
  __shared__ double red[32];
  const int K = 3 * Mx;
  const int a = blockIdx.x / K, b = blockIdx.x % K;
  double acc = 0.0;
  for (int i = threadIdx.x; i < nf; i += blockDim.x)
    acc += pair_col(UA, UB, MA, MB, Mx, nf, a, i) * pair_col(UA, UB, MA, MB, Mx, nf, b, i);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) G[blockIdx.x] = acc;
  }
}

// |u_A - u_B|^2 and |u_A|^2 (one CTA).  The difference of the two CP tensors is written
// as D * Mx terms whose factors are all small where the factor sets are close: per mode
// m, prod_d a_d - prod_d b_d = sum_k (prod_{d<k} b_d)(a_k - b_k)(prod_{d>k} a_d), so its
// squared norm, the sum over pairs of those terms of the products of their 1D inner
// products, keeps relative accuracy down to changes near the rounding of the factors
// (the expansion |a|^2 + |b|^2 - 2<a, b> cancels to ~sqrt(eps)).
__global__ void pair_change_kernel(const double* __restrict__ G, int D, int Mx, int MA, double* __restrict__ out) {
  __shared__ double rn[32], rd[32];
  double num = 0.0, den = 0.0;
  const int K = 3 * Mx, T = D * Mx;
  const size_t KK = (size_t)K * K;
  const long long TT = (long long)T * T;
  for (long long e = threadIdx.x; e < TT; e += blockDim.x) {
    const int p = (int)(e / T), q = (int)(e % T);
    const int kp = p / Mx, mp = p % Mx, kq = q / Mx, mq = q % Mx;
    double prod = 1.0;
    for (int d = 0; d < D; ++d) {
      const int cp = (d < kp ? Mx : (d == kp ? 2 * Mx : 0)) + mp;
      const int cq = (d < kq ? Mx : (d == kq ? 2 * Mx : 0)) + mq;
      prod *= G[(size_t)d * KK + (size_t)cp * K + cq];
    }
    num += prod;
  }
  for (int e = threadIdx.x; e < MA * MA; e += blockDim.x) {
    const int a = e / MA, b = e % MA;
    double prod = 1.0;
    for (int d = 0; d < D; ++d) prod *= G[(size_t)d * KK + (size_t)a * K + b];
    den += prod;
  }
  for (int o = 16; o > 0; o >>= 1) {
    num += __shfl_down_sync(0xffffffffu, num, o);
    den += __shfl_down_sync(0xffffffffu, den, o);
  }
  if ((threadIdx.x & 31) == 0) {
    rn[threadIdx.x >> 5] = num;
    rd[threadIdx.x >> 5] = den;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    num = threadIdx.x < (blockDim.x >> 5) ? rn[threadIdx.x] : 0.0;
    den = threadIdx.x < (blockDim.x >> 5) ? rd[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      num += __shfl_down_sync(0xffffffffu, num, o);
      den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (threadIdx.x == 0) {
      out[0] = num;
      out[1] = den;
    }
  }
}

extern "C" int taps_factors_rel_change(const taps_factors* A, const taps_factors* B, double* out) {
  if (!A || !B || !out || A->prob != B->prob || A->M < 1 || B->M < 1) return TAPS_ERR_INVALID_ARG;
  const taps_problem* P = A->prob;
  const int Mx = std::max(A->M, B->M), K = 3 * Mx, D = P->D;
  const size_t KK = (size_t)K * K;
  double* buf = nullptr;
  TAPS_TRY(taps_alloc((void**)&buf, sizeof(double) * (D * KK + 2)));
  int st = TAPS_OK;
  for (int d = 0; d < D && st == TAPS_OK; ++d) {
    pair_gram_kernel<<<(unsigned)KK, 128, 0, P->stream>>>(A->d_U[d], B->d_U[d], P->dims[d]->nf, A->M, B->M, Mx,
                                                           buf + (size_t)d * KK);
    if (cudaGetLastError() != cudaSuccess) st = TAPS_ERR_CUDA;
  }
  double h[2] = {0.0, 0.0};
  if (st == TAPS_OK) {
    pair_change_kernel<<<1, 1024, 0, P->stream>>>(buf, D, Mx, A->M, buf + (size_t)D * KK);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(h, buf + (size_t)D * KK, sizeof(h), cudaMemcpyDeviceToHost, P->stream) != cudaSuccess ||
        cudaStreamSynchronize(P->stream) != cudaSuccess)
      st = TAPS_ERR_CUDA;
  }
  cudaFree(buf);
  if (st != TAPS_OK) return st;
  *out = h[1] > 0.0 ? sqrt(std::max(h[0], 0.0) / h[1]) : 0.0;
  return TAPS_OK;
}

extern "C" const double* taps_factors_device_ptr(const taps_factors* U, int d) {
  if (!U || d < 0 || d >= U->prob->D) return nullptr;
  return U->d_U[d];
}

// Columns [m0, m1) of U_d by the init rule (SplitMix64 draws or zero/one).
// Columns m0..m1-1 of every dim's factor in one launch (thread per entry; the dims'
// entries one after another).
struct InitCols {
  double* U[TAPS_MAX_DIMS];
  long long off[TAPS_MAX_DIMS + 1];   // prefix of nf_d (m1 - m0)
  int nf[TAPS_MAX_DIMS];
  int D;
};

__global__ void init_cols_kernel(InitCols ic, int m0, int m1, int kind, unsigned seed) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ic.off[ic.D]) return;
  int d = 0;
  while (d + 1 < ic.D && idx >= ic.off[d + 1]) ++d;
  const long long loc = idx - ic.off[d];
  const int nf = ic.nf[d];
  int i = loc % nf, m = m0 + (int)(loc / nf);
  double v;
  if (kind == TAPS_INIT_RANDOM) v = taps_uniform_pm1(seed, d, i, m);
  else v = (d == 0) ? 0.0 : 1.0;
  ic.U[d][(size_t)m * nf + i] = v;
}

static int init_columns(taps_problem* P, taps_factors* U, int m0, int m1, int kind, unsigned seed) {
  if (m1 <= m0) return TAPS_OK;
  InitCols ic;
  memset(&ic, 0, sizeof(ic));
  ic.D = P->D;
  for (int d = 0; d < P->D; ++d) {
    ic.U[d] = U->d_U[d];
    ic.nf[d] = P->dims[d]->nf;
    ic.off[d + 1] = ic.off[d] + (long long)ic.nf[d] * (m1 - m0);
  }
  const long long tot = ic.off[P->D];
  int tk = prof_begin(P, TAPS_PROF_OTHER);
  init_cols_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, P->stream>>>(ic, m0, m1, kind, seed);
  prof_end(P, TAPS_PROF_OTHER, tk, 0.0, 8.0 * tot);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

// ---------------------------------------------------------------------------------
// Sweeps, residuals, solve
// ---------------------------------------------------------------------------------
static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

extern "C" int taps_sweep(taps_problem* P, taps_factors* U, int n_sweeps, const taps_sweep_opts* opts,
                          taps_sweep_report* rep) {
  if (!P || !U || U->prob != P || n_sweeps < 0 || U->M < 1) return TAPS_ERR_INVALID_ARG;
  int precision = opts ? opts->precision : TAPS_FP64;
  int solver = opts ? opts->solver : TAPS_SOLVER_BLOCK_LU;
  int normalize = opts ? opts->normalize : 1;
  if (precision < TAPS_FP64 || precision > TAPS_BF16) return TAPS_ERR_INVALID_ARG;
  if (solver < TAPS_SOLVER_BLOCK_LU || solver > TAPS_SOLVER_MODEDIAG) return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_weighted_ready(P));
  double t0 = now_s();
  TAPS_TRY(taps_ws_ensure(P, U->M));
  TAPS_TRY(taps_md_reset(P));
  TAPS_TRY(taps_refresh_grams(P, U, precision));
  double change = 0.0;
  for (int it = 0; it < n_sweeps; ++it) TAPS_TRY(taps_sweep_impl(P, U, precision, solver, normalize, &change));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  prof_drain(P);
  if (rep) {
    rep->sweeps = n_sweeps;
    rep->change = change;
    rep->seconds = now_s() - t0;
  }
  return TAPS_OK;
}

extern "C" int taps_residual(taps_problem* P, const taps_factors* U, int kind, double* rho_out) {
  if (!P || !U || !rho_out || U->prob != P || U->M < 1) return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_weighted_ready(P));
  return taps_residual_impl(P, U, kind, rho_out);
}

extern "C" int taps_solve(taps_problem* P, taps_factors* U, const taps_solve_opts* o,
                          taps_solve_report* rep) {
  if (!P || !U || !o || U->prob != P) return TAPS_ERR_INVALID_ARG;
  if (o->M_max < 1 || o->M_max > U->M_cap || o->max_sweeps < 1 ||
      o->precision < TAPS_FP64 || o->precision > TAPS_BF16 ||
      (o->res_kind != TAPS_RES_ALS && o->res_kind != TAPS_RES_FULL) ||
      o->init < TAPS_INIT_GIVEN || o->init > TAPS_INIT_ZERO ||
      o->solver < TAPS_SOLVER_BLOCK_LU || o->solver > TAPS_SOLVER_MODEDIAG)
    return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_weighted_ready(P));
  double t0 = now_s();
  if (o->init != TAPS_INIT_GIVEN) {
    if (o->M0 < 1 || o->M0 > o->M_max) return TAPS_ERR_INVALID_ARG;
    TAPS_TRY(init_columns(P, U, 0, o->M0, o->init, o->seed));
    U->M = o->M0;
  } else if (U->M < 1) {
    return TAPS_ERR_INVALID_ARG;
  }
  int add_kind = (o->init == TAPS_INIT_GIVEN) ? TAPS_INIT_RANDOM : o->init;
  int M = U->M;
  TAPS_TRY(taps_ws_ensure(P, o->M_max));
  TAPS_TRY(taps_md_reset(P));
  int precision = o->precision;
  TAPS_TRY(taps_refresh_grams(P, U, precision));
  int sweeps = 0, fp64_sweeps = 0, polish_left = o->polish_sweeps, hist = 0;
  double rho = INFINITY, change = INFINITY;
  bool converged = false;
  const int step = o->M_step > 0 ? o->M_step : 1;
  double rho_prev_M = INFINITY;   // residual at the end of the previous mode count
  int stalls = 0;
  // end of a mode count: true when the greedy growth stops on stagnation
  auto stalled = [&]() {
    if (!(o->res_stall > 0.0)) return false;
    const bool st = !(rho <= (1.0 - o->res_stall) * rho_prev_M);
    stalls = st ? stalls + 1 : 0;
    rho_prev_M = rho;
    return stalls >= 2;
  };
  while (true) {
    double prev_rho = INFINITY;
    int prec = precision;
    // FP64 / MIXED with graphs and the Eq. 42 residual: the whole sweep loop of this M
    // on the device (no host round trip per sweep)
    if (o->graphs == 2 && !taps_low_prec(prec) && o->res_kind == TAPS_RES_ALS && !P->prof->events) {
      int done = 0, fallback = 0;
      const double* dh = nullptr;
      const int lst = loop_solve(P, U, prec, o->solver, o->res_tol, o->als_tol, o->max_sweeps, &done, &dh, &fallback);
      if (!fallback) {
        for (int j = 0; j < done; ++j) {
          ++sweeps;
          if (prec == TAPS_FP64) ++fp64_sweeps;
          rho = dh[2 * j];
          change = dh[2 * j + 1];
          if (o->history_cap > 0 && rep && hist < o->history_cap) {
            if (rep->hist_M) rep->hist_M[hist] = M;
            if (rep->hist_change) rep->hist_change[hist] = change;
            if (rep->hist_rho) rep->hist_rho[hist] = rho;
            ++hist;
          }
        }
        TAPS_TRY(lst);
        if (rho <= o->res_tol) converged = true;
        if (converged || M >= o->M_max || stalled()) break;
        const int Mn = std::min(o->M_max, M + step);
        TAPS_TRY(init_columns(P, U, M, Mn, add_kind, o->seed));
        U->M = M = Mn;
        TAPS_TRY(taps_refresh_grams(P, U, precision));
        continue;
      }
    }
    for (int it = 0; it < o->max_sweeps; ++it) {
      if (taps_low_prec(prec)) {
        for (int d = 0; d < P->D; ++d)
          TAPS_CUDA(cudaMemcpyAsync(P->d_Usnap[d], U->d_U[d], sizeof(double) * P->dims[d]->nf * M,
                                    cudaMemcpyDeviceToDevice, P->stream));
      }
      int sst = TAPS_ERR_CUDA, fallback = 1;
      bool rho_done = false;
      if (o->graphs) {
        sst = graph_sweep(P, U, prec, o->solver, o->res_kind, &change, &rho, &fallback);
        rho_done = (sst == TAPS_OK);
      }
      if (fallback) sst = taps_sweep_impl(P, U, prec, o->solver, 1, &change);
      if (taps_low_prec(prec) && (sst == TAPS_ERR_SINGULAR || sst == TAPS_ERR_NONFINITE)) {
        // FP32 Grams cannot separate modes that agree to ~1e-8 (a Gram entry rounds to
        // an exact duplicate): restore the factors and redo the sweep in FP64.
        for (int d = 0; d < P->D; ++d)
          TAPS_CUDA(cudaMemcpyAsync(U->d_U[d], P->d_Usnap[d], sizeof(double) * P->dims[d]->nf * M,
                                    cudaMemcpyDeviceToDevice, P->stream));
        prec = TAPS_FP64;
        TAPS_TRY(taps_refresh_grams(P, U, TAPS_FP64));
        sst = taps_sweep_impl(P, U, prec, o->solver, 1, &change);
        rho_done = false;
      }
      TAPS_TRY(sst);
      ++sweeps;
      if (prec == TAPS_FP64) ++fp64_sweeps;
      if (!rho_done) TAPS_TRY(taps_residual_impl(P, U, o->res_kind, &rho, !taps_low_prec(prec)));
      if (o->history_cap > 0 && rep && hist < o->history_cap) {
        if (rep->hist_M) rep->hist_M[hist] = M;
        if (rep->hist_change) rep->hist_change[hist] = change;
        if (rep->hist_rho) rep->hist_rho[hist] = rho;
        ++hist;
      }
      if (rho <= o->res_tol) { converged = true; break; }
      if (change <= o->als_tol) break;
      if (taps_low_prec(prec)) {
        // FP32 / BF16 Grams stop helping once the residual no longer falls: refine in FP64.
        // If the FP32 sweep made the residual grow (an ill-conditioned factor set
        // amplifies single-precision Gram errors), go back to the pre-sweep factors.
        if (rho > 0.5 * prev_rho) {
          if (rho > prev_rho && std::isfinite(prev_rho)) {
            for (int d = 0; d < P->D; ++d)
              TAPS_CUDA(cudaMemcpyAsync(U->d_U[d], P->d_Usnap[d], sizeof(double) * P->dims[d]->nf * M,
                                        cudaMemcpyDeviceToDevice, P->stream));
            TAPS_TRY(taps_refresh_grams(P, U, TAPS_FP64));
            rho = prev_rho;
          }
          if (polish_left <= 0) break;
          prec = TAPS_FP64;
        }
      } else if (taps_low_prec(precision)) {
        if (--polish_left <= 0) break;
      }
      prev_rho = rho;
    }
    if (converged || M >= o->M_max || stalled()) break;
    const int Mn = std::min(o->M_max, M + step);
    TAPS_TRY(init_columns(P, U, M, Mn, add_kind, o->seed));
    U->M = M = Mn;
    TAPS_TRY(taps_refresh_grams(P, U, precision));
  }
  double rho_full = rho;
  if (o->res_kind != TAPS_RES_FULL) TAPS_TRY(taps_residual_impl(P, U, TAPS_RES_FULL, &rho_full));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  prof_drain(P);
  if (rep) {
    rep->M = M;
    rep->sweeps = sweeps;
    rep->fp64_sweeps = fp64_sweeps;
    rep->rho = rho;
    rep->rho_full = rho_full;
    rep->change = change;
    rep->seconds = now_s() - t0;
    rep->converged = converged ? 1 : 0;
    rep->hist_len = hist;
  }
  return converged ? TAPS_OK : TAPS_ERR_NOT_CONVERGED;
}

// ---------------------------------------------------------------------------------
// Grid reconstruction (Eq. 13 at nodes): u[i_1..i_D] = sum_m prod_d U_d[i_d, m].
// The dims are split into leading "row" dims and trailing "column" dims (at least
// 128 columns when the grid allows), so the output is the rank-M product
// out[r][c] = sum_m A[r][m] B[c][m] with A = row-wise products of the leading dims'
// factor rows and B = those of the trailing dims.  A and B are built by
// eval_factor_kernel; eval_gemm_kernel streams the output with register tiles.
// ---------------------------------------------------------------------------------

template <typename T>
__global__ void gather_rows_kernel(const double* U, int nf, int off, int start, int step, int count,
                                   int M, T* G) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count * M) return;
  int j = idx / M, m = idx % M;
  int node = start + step * j;
  int fj = node - off;
  G[idx] = (fj >= 0 && fj < nf) ? (T)U[(size_t)m * nf + fj] : (T)0;
}

// X[x][m] = prod_{d in [d0, d1)} G_d[i_d(x)][m], x in C order over dims d0..d1-1.
template <typename T>
__global__ void eval_factor_kernel(const T* __restrict__ G, GridSpec gs, int d0, int d1, int M,
                                   long long nx, T* __restrict__ X) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nx * M) return;
  long long x = idx / M;
  int m = (int)(idx - x * M);
  T v = (T)1;
  for (int d = d1 - 1; d >= d0; --d) {
    long long q = x / gs.count[d];
    int id = (int)(x - q * gs.count[d]);
    x = q;
    v *= G[gs.goff[d] + (long long)id * M + m];
  }
  X[idx] = v;
}

// out[r][c] = sum_m A[r][m] B[c][m].  CTA tile 128 x 128 (256 threads), thread tile
// 8 x 8 with rows ty + 16a and columns tx + 16b, so that shared-memory reads are
// broadcasts / conflict-free and every warp store covers two 64-byte row segments.
// The tiles are stored transposed ([m][row]) with a padded stride (129) so that the
// transposing fill is conflict-free.  The FP32 product uses packed fma.rn.f32x2.
#define EB 128
#define EBP 129

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}

template <typename T>
__device__ __forceinline__ void eval_fill(const T* __restrict__ A, const T* __restrict__ B, long long r0,
                                          int c0, int nr, int nc, int M, T* As, T* Bs) {
  for (int idx = threadIdx.x; idx < EB * M; idx += blockDim.x) {
    int r = idx / M, m = idx - r * M;
    As[m * EBP + r] = (r < nr) ? A[(r0 + r) * M + m] : (T)0;
    Bs[m * EBP + r] = (r < nc) ? B[(long long)(c0 + r) * M + m] : (T)0;
  }
}

__global__ void __launch_bounds__(256) eval_gemm_f32_kernel(const float* __restrict__ A,
                                                            const float* __restrict__ B, long long R,
                                                            int C, int M, float* __restrict__ out) {
  extern __shared__ __align__(16) float smf[];
  float* As = smf;              // [M][EBP]
  float* Bs = smf + M * EBP;    // [M][EBP]
  const long long r0 = (long long)blockIdx.x * EB;
  const int c0 = blockIdx.y * EB;
  const int nr = (int)min((long long)EB, R - r0);
  const int nc = min(EB, C - c0);
  eval_fill<float>(A, B, r0, c0, nr, nc, M, As, Bs);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  unsigned long long acc[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0ull;
  for (int m = 0; m < M; ++m) {
    const float* ar = As + m * EBP + ty;
    const float* br = Bs + m * EBP + tx;
    unsigned long long bv[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) bv[b] = pack2(br[32 * b], br[32 * b + 16]);
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      float av = ar[16 * a];
      unsigned long long aa = pack2(av, av);
#pragma unroll
      for (int b = 0; b < 4; ++b) asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(acc[a][b]) : "l"(aa), "l"(bv[b]));
    }
  }
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    int r = ty + 16 * a;
    if (r >= nr) continue;
    float* o = out + (r0 + r) * (long long)C + c0 + tx;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      float lo, hi;
      unpack2(acc[a][b], lo, hi);
      if (tx + 32 * b < nc) __stcs(o + 32 * b, lo);
      if (tx + 32 * b + 16 < nc) __stcs(o + 32 * b + 16, hi);
    }
  }
}

__global__ void __launch_bounds__(256) eval_gemm_f64_kernel(const double* __restrict__ A,
                                                            const double* __restrict__ B, long long R,
                                                            int C, int M, double* __restrict__ out) {
  extern __shared__ __align__(16) double smd[];
  double* As = smd;
  double* Bs = smd + M * EBP;
  const long long r0 = (long long)blockIdx.x * EB;
  const int c0 = blockIdx.y * EB;
  const int nr = (int)min((long long)EB, R - r0);
  const int nc = min(EB, C - c0);
  eval_fill<double>(A, B, r0, c0, nr, nc, M, As, Bs);
  __syncthreads();
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
  for (int half = 0; half < 2; ++half) {  // 4 of the 8 rows per pass keeps registers bounded
    double acc[4][8];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.0;
    for (int m = 0; m < M; ++m) {
      double av[4], bv[8];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[m * EBP + ty + 16 * (4 * half + a)];
#pragma unroll
      for (int b = 0; b < 8; ++b) bv[b] = Bs[m * EBP + tx + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 8; ++b) acc[a][b] += av[a] * bv[b];
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      int r = ty + 16 * (4 * half + a);
      if (r >= nr) continue;
      double* o = out + (r0 + r) * (long long)C + c0 + tx;
#pragma unroll
      for (int b = 0; b < 8; ++b)
        if (tx + 16 * b < nc) o[16 * b] = acc[a][b];
    }
  }
}

extern "C" int taps_eval_grid(const taps_problem* Pc, const taps_factors* U, const int* start,
                              const int* count, const int* step, void* out_dev, int out_dtype) {
  taps_problem* P = const_cast<taps_problem*>(Pc);
  if (!P || !U || !start || !count || !step || U->M < 1) return TAPS_ERR_INVALID_ARG;
  if (out_dtype != TAPS_FP64 && out_dtype != TAPS_FP32) return TAPS_ERR_INVALID_ARG;
  GridSpec gs;
  memset(&gs, 0, sizeof(gs));
  gs.D = P->D;
  long long total = 1, goff = 0;
  int M = U->M;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    if (count[d] < 1) return TAPS_ERR_INVALID_ARG;
    long long first = start[d], lastn = start[d] + (long long)step[d] * (count[d] - 1);
    if (first < 0 || first >= dm->n || lastn < 0 || lastn >= dm->n) return TAPS_ERR_INVALID_ARG;
    gs.count[d] = count[d];
    gs.goff[d] = goff;
    goff += (long long)count[d] * M;
    total *= count[d];
  }
  if (!out_dev) return TAPS_ERR_INVALID_ARG;
  cudaStream_t s = P->stream;
  size_t esz = out_dtype == TAPS_FP64 ? sizeof(double) : sizeof(float);
  int st = TAPS_OK;
  int split = P->D - 1;
  long long cols = count[P->D - 1];
  while (split > 1 && cols < 128) cols *= count[--split];
  if (cols > (1ll << 30)) return TAPS_ERR_INVALID_ARG;
  long long rows = total / cols;
  const bool use_tc = out_dtype == TAPS_FP32 && taps_eval_tc_usable(rows, cols, M);
  const size_t gbytes = (esz * (size_t)goff + 255) / 256 * 256;
  size_t need = use_tc ? gbytes + taps_eval_tc_scratch(rows, cols, M) : esz * (goff + (size_t)(rows + cols) * M);
  if (need > P->evalbuf_len) {
    TAPS_CUDA(cudaStreamSynchronize(s));
    cudaFree(P->d_evalbuf);
    P->d_evalbuf = nullptr;
    P->evalbuf_len = 0;
    TAPS_TRY(taps_alloc(&P->d_evalbuf, need));
    P->evalbuf_len = need;
  }
  void* G = P->d_evalbuf;
  if (!P->eval_attr_set) {
    int dev = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    TAPS_CUDA(cudaFuncSetAttribute((const void*)eval_gemm_f64_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    TAPS_CUDA(cudaFuncSetAttribute((const void*)eval_gemm_f32_kernel,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm));
    TAPS_TRY(taps_eval_tc_setup(maxsm));
    P->eval_attr_set = 1;
  }
  int tk = prof_begin(P, TAPS_PROF_EVAL);
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    int n = count[d] * M;
    if (out_dtype == TAPS_FP64)
      gather_rows_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(U->d_U[d], dm->nf, dm->off, start[d],
                                                                 step[d], count[d], M,
                                                                 (double*)G + gs.goff[d]);
    else
      gather_rows_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(U->d_U[d], dm->nf, dm->off, start[d],
                                                                step[d], count[d], M,
                                                                (float*)G + gs.goff[d]);
  }
  if (use_tc) {
    st = taps_eval_tc(P, (const float*)G, gs, split, M, rows, cols, (char*)G + gbytes, (float*)out_dev);
    if (st != TAPS_OK) return st;
  } else if (out_dtype == TAPS_FP64) {
    double* A = (double*)G + goff;
    double* B = A + rows * M;
    eval_factor_kernel<double><<<(unsigned)((rows * M + 255) / 256), 256, 0, s>>>((const double*)G, gs, 0, split, M, rows, A);
    eval_factor_kernel<double><<<(unsigned)((cols * M + 255) / 256), 256, 0, s>>>((const double*)G, gs, split, P->D, M, cols, B);
    dim3 eg((unsigned)((rows + EB - 1) / EB), (unsigned)((cols + EB - 1) / EB));
    eval_gemm_f64_kernel<<<eg, 256, (size_t)M * 2 * EBP * sizeof(double), s>>>(A, B, rows, (int)cols, M, (double*)out_dev);
  } else {
    float* A = (float*)G + goff;
    float* B = A + rows * M;
    eval_factor_kernel<float><<<(unsigned)((rows * M + 255) / 256), 256, 0, s>>>((const float*)G, gs, 0, split, M, rows, A);
    eval_factor_kernel<float><<<(unsigned)((cols * M + 255) / 256), 256, 0, s>>>((const float*)G, gs, split, P->D, M, cols, B);
    dim3 eg((unsigned)((rows + EB - 1) / EB), (unsigned)((cols + EB - 1) / EB));
    eval_gemm_f32_kernel<<<eg, 256, (size_t)M * 2 * EBP * sizeof(float), s>>>(A, B, rows, (int)cols, M, (float*)out_dev);
  }
  P->prof->launches[TAPS_PROF_EVAL] += P->D + 2;  // gathers, two factor products / images, product
  prof_end(P, TAPS_PROF_EVAL, tk, 2.0 * M * (double)total + (double)(rows + cols) * M * (P->D - 1),
           (double)esz * total);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    taps_note_cuda_error(e, "eval_grid_kernel", __FILE__, __LINE__);
    st = TAPS_ERR_CUDA;
  }
  return st;
}


// ---------------------------------------------------------------------------------
// Batched independent instances: one sweep of every instance captured as one CUDA
// graph (each instance on its own stream, forked from and joined to a master stream),
// replayed n_sweeps times back to back.  Without graphs each instance runs its own
// launch sequence in turn (the one-launch-sequence-per-instance baseline).
// ---------------------------------------------------------------------------------
struct taps_batch {
  int count, precision, solver;
  int eff_solver;     // the solver the sweeps use (AUTO: the tuner's choice)
  int tuned;
  float trial_ms[2];  // AUTO: one graph sweep with FASTDIAG, with MODEDIAG
  taps_problem** P;
  taps_factors** U;
  cudaStream_t master;
  cudaEvent_t fork;
  cudaEvent_t* join;
  cudaGraph_t g;
  cudaGraphExec_t exec;
  // batched tensor-core Gram refresh: queue buffer, per-item tickets, the tile choice
  // (chunk rows, CTAs per SM) of the tuner and its trial times
  void* gt_buf;
  size_t gt_buf_bytes;
  double* gt_partial;
  size_t gt_partial_len;
  unsigned* gt_tickets;
  int gt_items_cap;
  int gt_rows, gt_cps, gt_tuned;
  float gt_table[6];
};

extern "C" void taps_batch_destroy(taps_batch* B) {
  if (!B) return;
  if (B->master) cudaStreamSynchronize(B->master);
  if (B->gt_buf) cudaFree(B->gt_buf);
  if (B->gt_partial) cudaFree(B->gt_partial);
  if (B->gt_tickets) cudaFree(B->gt_tickets);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->g) cudaGraphDestroy(B->g);
  if (B->join) {
    for (int i = 0; i < B->count; ++i) cudaEventDestroy(B->join[i]);
    delete[] B->join;
  }
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->master) cudaStreamDestroy(B->master);
  delete[] B->P;
  delete[] B->U;
  delete B;
}

extern "C" int taps_batch_create(taps_problem* const* probs, taps_factors* const* Us, int count, int precision,
                                 int solver, taps_batch** out) {
  if (!probs || !Us || !out || count < 1 || (precision != TAPS_FP64 && precision != TAPS_MIXED) ||
      solver < TAPS_SOLVER_BLOCK_LU || solver > TAPS_SOLVER_AUTO)
    return TAPS_ERR_INVALID_ARG;
  *out = nullptr;
  for (int i = 0; i < count; ++i) {
    if (!probs[i] || !Us[i] || Us[i]->prob != probs[i] || Us[i]->M < 1) return TAPS_ERR_INVALID_ARG;
    if (taps_weighted_ready(probs[i]) != TAPS_OK) return TAPS_ERR_INVALID_ARG;
    for (int j = 0; j < i; ++j)
      if (probs[j] == probs[i]) return TAPS_ERR_INVALID_ARG;   // instances must not share workspaces
  }
  taps_batch* B = new taps_batch();
  memset((void*)B, 0, sizeof(taps_batch));
  B->count = count;
  B->precision = precision;
  B->solver = solver;
  B->eff_solver = solver == TAPS_SOLVER_AUTO ? TAPS_SOLVER_FASTDIAG : solver;
  B->P = new taps_problem*[count];
  B->U = new taps_factors*[count];
  for (int i = 0; i < count; ++i) { B->P[i] = probs[i]; B->U[i] = Us[i]; }
  int st = TAPS_OK;
  do {
    if (cudaStreamCreateWithFlags(&B->master, cudaStreamNonBlocking) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    B->join = new cudaEvent_t[count];
    memset(B->join, 0, sizeof(cudaEvent_t) * count);
    for (int i = 0; i < count && st == TAPS_OK; ++i)
      if (cudaEventCreateWithFlags(&B->join[i], cudaEventDisableTiming) != cudaSuccess) st = TAPS_ERR_CUDA;
    // pencil decompositions in waves of instances, each instance on its own stream,
    // so that the small-grid kernels of different instances share the GPU
    const int wave = 32;
    std::vector<FdPending> pend;
    for (int i0 = 0; i0 < count && st == TAPS_OK; i0 += wave) {
      const int i1 = std::min(count, i0 + wave);
      for (int i = i0; i < i1 && st == TAPS_OK; ++i) {
        if ((st = taps_ws_ensure(B->P[i], B->U[i]->M)) != TAPS_OK) break;
        // FASTDIAG's pencils cover MODEDIAG's (the dims it cannot solve on the mode side)
        st = taps_fd_prepare_enqueue(B->P[i], B->eff_solver, B->U[i]->M, &pend);
      }
      int s2 = taps_fd_prepare_finish(&pend);
      if (st == TAPS_OK) st = s2;
    }
    for (int i = 0; i < count && st == TAPS_OK; ++i) {
      taps_problem* P = B->P[i];
      if ((st = taps_refresh_grams(P, B->U[i], TAPS_FP64)) != TAPS_OK) break;
    }
    for (int i = 0; i < count && st == TAPS_OK; ++i)
      if (cudaStreamSynchronize(B->P[i]->stream) != cudaSuccess) st = TAPS_ERR_CUDA;
  } while (0);
  if (st != TAPS_OK) {
    taps_batch_destroy(B);
    return st;
  }
  *out = B;
  return TAPS_OK;
}

static int batch_capture(taps_batch* B) {
  if (B->exec) return TAPS_OK;
  if (cudaStreamBeginCapture(B->master, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TAPS_ERR_CUDA;
  int st = TAPS_OK;
  cudaEventRecord(B->fork, B->master);
  cudaStream_t* saved = new cudaStream_t[B->count];
  for (int i = 0; i < B->count; ++i) {
    taps_problem* P = B->P[i];
    saved[i] = P->stream;
    P->stream = P->cap_stream;
    bool cap = P->prof->capturing;
    P->prof->capturing = true;    // no event-pool growth or synchronisation inside capture
    cudaStreamWaitEvent(P->cap_stream, B->fork, 0);
    // the batch graph replays after batched Gram refreshes too: it forms dim 0's
    // coefficients itself
    const int c0_before = P->c0_valid, c0_M_before = P->c0_M;
    P->c0_forbid = 1;
    if (st == TAPS_OK) st = taps_sweep_enqueue(P, B->U[i], B->precision, B->eff_solver, 1);
    P->c0_forbid = 0;
    P->c0_valid = c0_before;
    P->c0_M = c0_M_before;
    cudaEventRecord(B->join[i], P->cap_stream);
    cudaStreamWaitEvent(B->master, B->join[i], 0);
    P->prof->capturing = cap;
  }
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(B->master, &g);
  for (int i = 0; i < B->count; ++i) {
    B->P[i]->stream = saved[i];
    // events recorded inside the batch graph stay owned by the graph's lifetime; the
    // instances' pending lists are cleared (their timing is not read for batches)
    B->P[i]->prof->npending = 0;
  }
  delete[] saved;
  if (ce != cudaSuccess || !g) {
    cudaGetLastError();
    return st != TAPS_OK ? st : TAPS_ERR_CUDA;
  }
  B->g = g;
  if (st == TAPS_OK && cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    st = TAPS_ERR_CUDA;
  }
  return st;
}

static void batch_drop_graph(taps_batch* B) {
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->g) cudaGraphDestroy(B->g);
  B->exec = nullptr;
  B->g = nullptr;
}

// Joins every instance's stream into the batch's stream.
static int batch_join(taps_batch* B) {
  for (int i = 0; i < B->count; ++i) {
    TAPS_CUDA(cudaEventRecord(B->join[i], B->P[i]->stream));
    TAPS_CUDA(cudaStreamWaitEvent(B->master, B->join[i], 0));
  }
  return TAPS_OK;
}

// TAPS_SOLVER_AUTO: one graph sweep of the whole batch with each candidate solver,
// timed with events on the batch's stream; every instance's factors, Grams and status
// are restored after each trial.  The faster candidate is kept.
static int batch_autotune(taps_batch* B) {
  size_t tot = 0;
  for (int i = 0; i < B->count; ++i)
    for (int d = 0; d < B->P[i]->D; ++d) tot += (size_t)B->P[i]->dims[d]->nf * B->U[i]->M;
  double* backup = nullptr;
  TAPS_TRY(taps_alloc((void**)&backup, sizeof(double) * std::max(tot, (size_t)1)));
  auto copy_all = [&](bool save) -> int {
    size_t off = 0;
    for (int i = 0; i < B->count; ++i)
      for (int d = 0; d < B->P[i]->D; ++d) {
        const size_t len = (size_t)B->P[i]->dims[d]->nf * B->U[i]->M;
        double* dev = B->U[i]->d_U[d];
        TAPS_CUDA(cudaMemcpyAsync(save ? backup + off : dev, save ? dev : backup + off, sizeof(double) * len,
                                  cudaMemcpyDeviceToDevice, B->P[i]->stream));
        off += len;
      }
    return TAPS_OK;
  };
  const int cands[2] = {TAPS_SOLVER_FASTDIAG, TAPS_SOLVER_MODEDIAG};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int st = TAPS_OK, best = TAPS_SOLVER_FASTDIAG;
  float best_ms = 1e30f;
  do {
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    if ((st = copy_all(true)) != TAPS_OK) break;
    for (int k = 0; k < 2 && st == TAPS_OK; ++k) {
      batch_drop_graph(B);
      B->eff_solver = cands[k];
      if ((st = batch_capture(B)) != TAPS_OK) break;
      if (cudaGraphUpload(B->exec, B->master) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
      if ((st = batch_join(B)) != TAPS_OK) break;
      cudaEventRecord(e0, B->master);
      if (cudaGraphLaunch(B->exec, B->master) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
      cudaEventRecord(e1, B->master);
      if (cudaEventSynchronize(e1) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      B->trial_ms[k] = ms;
      if (ms < best_ms) {
        best_ms = ms;
        best = cands[k];
      }
      for (int i = 0; i < B->count; ++i) {   // consume the trial's status words
        double ch = 0.0;
        if (taps_sweep_finish(B->P[i], B->U[i], &ch) == TAPS_ERR_CUDA) st = TAPS_ERR_CUDA;
      }
      if (st != TAPS_OK || (st = copy_all(false)) != TAPS_OK) break;
      for (int i = 0; i < B->count && st == TAPS_OK; ++i) {
        if ((st = taps_md_reset(B->P[i])) == TAPS_OK) st = taps_refresh_grams(B->P[i], B->U[i], TAPS_FP64);
      }
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  for (int i = 0; i < B->count; ++i) cudaStreamSynchronize(B->P[i]->stream);
  cudaFree(backup);
  if (st != TAPS_OK) return st;
  if (B->eff_solver != best) {
    batch_drop_graph(B);
    B->eff_solver = best;
  }
  B->tuned = 1;
  return TAPS_OK;
}

extern "C" int taps_batch_info(const taps_batch* B, int* solver_out, float* trial_ms_out) {
  if (!B) return TAPS_ERR_INVALID_ARG;
  if (solver_out) *solver_out = B->eff_solver;
  if (trial_ms_out) {
    trial_ms_out[0] = B->tuned ? B->trial_ms[0] : -1.f;
    trial_ms_out[1] = B->tuned ? B->trial_ms[1] : -1.f;
  }
  return TAPS_OK;
}

extern "C" int taps_batch_sweep(taps_batch* B, int n_sweeps, int graphs, double* changes_out, int* status_out) {
  if (!B || n_sweeps < 1) return TAPS_ERR_INVALID_ARG;
  if (graphs && B->solver == TAPS_SOLVER_AUTO && !B->tuned) TAPS_TRY(batch_autotune(B));
  // the factors may have been set since the last call: every instance's Grams are
  // recomputed from its current factors first (as taps_sweep does)
  for (int i = 0; i < B->count; ++i) {
    TAPS_TRY(taps_md_reset(B->P[i]));
    TAPS_TRY(taps_refresh_grams(B->P[i], B->U[i], TAPS_FP64));
  }
  int first = TAPS_OK;
  auto note = [&](int i, int st, double ch) {
    if (changes_out) changes_out[i] = ch;
    if (status_out) status_out[i] = st;
    if (first == TAPS_OK) first = st;
  };
  if (graphs) {
    TAPS_TRY(batch_capture(B));
    TAPS_TRY(batch_join(B));
    for (int it = 0; it < n_sweeps; ++it) TAPS_CUDA(cudaGraphLaunch(B->exec, B->master));
    TAPS_CUDA(cudaStreamSynchronize(B->master));
    for (int i = 0; i < B->count; ++i) {
      double ch = 0.0;
      const int st = taps_sweep_finish(B->P[i], B->U[i], &ch);
      if (st == TAPS_ERR_CUDA) return st;
      note(i, st, st == TAPS_OK ? ch : NAN);
    }
  } else {
    for (int i = 0; i < B->count; ++i) {
      double ch = 0.0;
      int sti = TAPS_OK;
      for (int it = 0; it < n_sweeps; ++it) {   // all sweeps run, as in the graph
        const int st = taps_sweep_impl(B->P[i], B->U[i], B->precision, B->eff_solver, 1, &ch);
        if (st == TAPS_ERR_CUDA) return st;
        if (sti == TAPS_OK) sti = st;
      }
      note(i, sti, sti == TAPS_OK ? ch : NAN);
    }
  }
  return status_out ? TAPS_OK : first;
}

// ---------------------------------------------------------------------------------
// Gram refresh of every dim of every instance of a batch in one persistent launch
// (tensor cores, BF16 operands) or instance by instance (FP64, CUDA cores).
// ---------------------------------------------------------------------------------
#define GT_CAND 6
#define GT_CPT 8   // chunks per task of the batched Gram refresh
static const int kGtRows[GT_CAND] = {64, 64, 64, 64, 128, 128};
static const int kGtCps[GT_CAND] = {1, 2, 3, 4, 1, 2};

extern "C" int taps_batch_refresh_grams(taps_batch* B, int precision, float* ms_out, double* bytes_out) {
  if (!B || (precision != TAPS_FP64 && precision != TAPS_BF16)) return TAPS_ERR_INVALID_ARG;
  std::vector<GtHostItem> items;
  int maxN = 16, maxNH = 16, maxops = 1;
  size_t chunks64 = 0, partial_need = 0;
  double bytes = 0.0;
  for (int i = 0; i < B->count; ++i) {
    taps_problem* P = B->P[i];
    taps_factors* U = B->U[i];
    for (int d = 0; d < P->D; ++d) {
      const taps_dim* dm = P->dims[d];
      GtHostItem h;
      h.U = U->d_U[d];
      h.band = P->d_opband[d];
      h.q = P->d_q[d];
      h.gram = P->d_gram[d];
      h.h = P->d_h[d];
      h.n = dm->nf;
      h.M = U->M;
      h.hb = dm->hb;
      h.nops = P->tt.nops[d];
      h.Rf = P->Rf;
      if (precision == TAPS_BF16 && !taps_gram_tc_eligible(h.M, h.nops, h.Rf, h.hb)) return TAPS_ERR_INVALID_ARG;
      items.push_back(h);
      maxN = std::max(maxN, (h.M + 15) & ~15);
      maxNH = std::max(maxNH, (h.Rf + 15) & ~15);
      maxops = std::max(maxops, h.nops);
      chunks64 += (size_t)(h.n + 63) / 64;
      // partial sums of an item split over tasks of GT_CPT chunks (64-node chunks: the most tasks)
      const size_t tasks64 = ((size_t)(h.n + 63) / 64 + GT_CPT - 1) / GT_CPT;
      if (tasks64 > 1) partial_need += tasks64 * ((size_t)h.nops * h.M * h.M + (size_t)h.Rf * h.M);
      const int nb = 2 * h.hb + 1;
      bytes += 8.0 * ((double)h.n * h.M + (double)h.nops * h.n * nb + (double)h.Rf * h.n +
                      (double)h.nops * h.M * h.M + (double)h.Rf * h.M);
    }
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  TAPS_CUDA(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return TAPS_ERR_CUDA;
  }
  int st = TAPS_OK;
  float ms = 0.f;
  do {
    if ((st = batch_join(B)) != TAPS_OK) break;
    if (precision == TAPS_FP64) {
      // instance by instance on their own streams, forked from and joined to the batch's
      if (cudaEventRecord(e0, B->master) != cudaSuccess || cudaEventRecord(B->fork, B->master) != cudaSuccess) {
        st = TAPS_ERR_CUDA;
        break;
      }
      for (int i = 0; i < B->count && st == TAPS_OK; ++i) {
        if (cudaStreamWaitEvent(B->P[i]->stream, B->fork, 0) != cudaSuccess) st = TAPS_ERR_CUDA;
        else st = taps_refresh_grams(B->P[i], B->U[i], TAPS_FP64);
      }
      if (st != TAPS_OK || (st = batch_join(B)) != TAPS_OK) break;
      if (cudaEventRecord(e1, B->master) != cudaSuccess) st = TAPS_ERR_CUDA;
    } else {
      const int dev_sms = B->P[0]->num_sms;
      for (int i = 0; i < B->count; ++i) B->P[i]->c0_valid = 0;   // Grams replaced, no coefficients formed
      const size_t need = taps_gram_tc_queue_bytes((int)items.size(), (int)chunks64);
      if (need > B->gt_buf_bytes) {
        if (B->gt_buf) cudaFree(B->gt_buf);
        B->gt_buf = nullptr;
        B->gt_buf_bytes = 0;
        if ((st = taps_alloc(&B->gt_buf, need)) != TAPS_OK) break;
        B->gt_buf_bytes = need;
      }
      if (partial_need > B->gt_partial_len) {
        if (B->gt_partial) cudaFree(B->gt_partial);
        B->gt_partial = nullptr;
        B->gt_partial_len = 0;
        if ((st = taps_alloc((void**)&B->gt_partial, sizeof(double) * partial_need)) != TAPS_OK) break;
        B->gt_partial_len = partial_need;
      }
      if ((int)items.size() > B->gt_items_cap) {
        if (B->gt_tickets) cudaFree(B->gt_tickets);
        B->gt_tickets = nullptr;
        B->gt_items_cap = 0;
        if ((st = taps_alloc((void**)&B->gt_tickets, sizeof(unsigned) * items.size())) != TAPS_OK) break;
        if (cudaMemsetAsync(B->gt_tickets, 0, sizeof(unsigned) * items.size(), B->master) != cudaSuccess) {
          st = TAPS_ERR_CUDA;
          break;
        }
        B->gt_items_cap = (int)items.size();
      }
      int* status = B->P[0]->d_status;
      // tasks of GT_CPT chunks (a dim of more than GT_CPT chunks is split, its partial
      // sums added in task order by its last task); the tuner times the chunk height and
      // the CTAs per SM the shared memory and TMEM allow
      if (!B->gt_tuned) {
        int maxsm = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
        float best = 1e30f;
        for (int k = 0; k < GT_CAND && st == TAPS_OK; ++k) {
          size_t smem = 0;
          int ncols = 0;
          taps_gram_tc_footprint(kGtRows[k], maxN, maxNH, maxops, &smem, &ncols);
          B->gt_table[k] = -1.f;
          if ((size_t)kGtCps[k] * (smem + 1024) > (size_t)maxsm || kGtCps[k] * ncols > 512) continue;
          st = taps_gram_tc_queue(items, kGtRows[k], GT_CPT, dev_sms * kGtCps[k], B->gt_buf, B->gt_buf_bytes,
                                  B->gt_partial, B->gt_partial_len, B->gt_tickets, B->master, status, nullptr,
                                  nullptr, e0, e1);
          if (st != TAPS_OK) break;
          float t = 0.f;
          cudaEventElapsedTime(&t, e0, e1);
          B->gt_table[k] = t;
          if (t < best) {
            best = t;
            B->gt_rows = kGtRows[k];
            B->gt_cps = kGtCps[k];
          }
        }
        if (st != TAPS_OK) break;
        B->gt_tuned = 1;
      }
      st = taps_gram_tc_queue(items, B->gt_rows, GT_CPT, dev_sms * B->gt_cps, B->gt_buf, B->gt_buf_bytes,
                              B->gt_partial, B->gt_partial_len, B->gt_tickets, B->master, status, nullptr, nullptr,
                              e0, e1);
      if (st != TAPS_OK) break;
    }
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      st = TAPS_ERR_CUDA;
      break;
    }
    cudaEventElapsedTime(&ms, e0, e1);
    // the instances' next work sees the new Grams
    if (cudaEventRecord(B->fork, B->master) != cudaSuccess) st = TAPS_ERR_CUDA;
    for (int i = 0; i < B->count && st == TAPS_OK; ++i)
      if (cudaStreamWaitEvent(B->P[i]->stream, B->fork, 0) != cudaSuccess) st = TAPS_ERR_CUDA;
    if (st == TAPS_OK) st = taps_check_status(B->P[0]->d_status, B->master);
  } while (0);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != TAPS_OK) return st;
  if (ms_out) *ms_out = ms;
  if (bytes_out) *bytes_out = bytes;
  return TAPS_OK;
}

extern "C" int taps_batch_gram_info(const taps_batch* B, int* rows_out, int* ctas_per_sm_out, float* table_ms_out) {
  if (!B) return TAPS_ERR_INVALID_ARG;
  if (rows_out) *rows_out = B->gt_tuned ? B->gt_rows : 0;
  if (ctas_per_sm_out) *ctas_per_sm_out = B->gt_tuned ? B->gt_cps : 0;
  if (table_ms_out)
    for (int k = 0; k < GT_CAND; ++k) table_ms_out[k] = B->gt_tuned ? B->gt_table[k] : -1.f;
  return TAPS_OK;
}

extern "C" int taps_problem_refresh_grams(taps_problem* P, const taps_factors* U, int precision) {
  if (!P || !U || U->prob != P || U->M < 1 ||
      (precision != TAPS_FP64 && precision != TAPS_FP32 && precision != TAPS_BF16))
    return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_ws_ensure(P, U->M));
  TAPS_TRY(taps_refresh_grams(P, U, precision));
  return taps_check_status(P->d_status, P->stream);
}

extern "C" int taps_problem_copy_grams(const taps_problem* P, int d, int M, double* gram_out, double* h_out,
                                       int* ops_out, int* nops_out) {
  if (!P || d < 0 || d >= P->D || M < 1 || M > P->ws_M) return TAPS_ERR_INVALID_ARG;
  const int nops = P->tt.nops[d];
  if (nops_out) *nops_out = nops;
  if (ops_out)
    for (int o = 0; o < nops; ++o) ops_out[o] = P->ops[d][o];
  if (gram_out)
    TAPS_CUDA(cudaMemcpyAsync(gram_out, P->d_gram[d], sizeof(double) * nops * M * M, cudaMemcpyDeviceToHost,
                              P->stream));
  if (h_out)
    TAPS_CUDA(cudaMemcpyAsync(h_out, P->d_h[d], sizeof(double) * P->Rf * M, cudaMemcpyDeviceToHost, P->stream));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return TAPS_OK;
}
