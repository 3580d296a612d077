// Internal declarations shared by the TAPS CUDA translation units (GPU path only).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string.h>

#include <cmath>
#include <vector>

#include "taps.h"

#define TAPS_WARP 32

// Record a CUDA error and return TAPS_ERR_CUDA from the calling entry point.
#define TAPS_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) {                             \
      taps_note_cuda_error(e_, #call, __FILE__, __LINE__); \
      return TAPS_ERR_CUDA;                              \
    }                                                    \
  } while (0)

#define TAPS_TRY(expr)          \
  do {                          \
    int s_ = (expr);            \
    if (s_ != TAPS_OK) return s_; \
  } while (0)

void taps_note_cuda_error(cudaError_t e, const char* what, const char* file, int line);
int taps_alloc(void** p, size_t bytes);

// Device status word values (set with atomicCAS so the first error wins).
#define TAPS_DEV_OK 0
#define TAPS_DEV_SINGULAR 1
#define TAPS_DEV_NONFINITE 2
#define TAPS_DEV_TIMEOUT 3
int taps_status_from_device(int dev);

// Fast-diagonalisation data of one operator pencil (A, B) of a dimension:
// Phi^T B Phi = I, Phi^T A Phi = diag(mu) over the free nodes (A absent: opA = -1).
struct FdEntry {
  int opA, opB;
  int status;
  int pending;         // enqueued, not yet finished (done marks its last kernel)
  cudaEvent_t done;
  double* Phi;   // [nf][nf] row-major
  double* PhiT;  // [nf][nf] row-major (transpose)
  double* mu;    // [nf]
};

// ---------------------------------------------------------------------------------
// Assembled dimension: C-HiDeNN tables and banded 1D matrices on the device.
// ---------------------------------------------------------------------------------
struct taps_dim {
  taps_dim_desc desc;
  int n;        // all nodes
  int nf;       // free nodes
  int off;      // index of the first free node (1 with a Dirichlet low end)
  int hb;       // band half-width 2s+1
  int nb;       // band width 2hb+1
  int amax;     // max patch size 2s+1
  int pmax;     // moment-matrix size 2s+1+p+1
  int nloc;     // nodes touching one element 2s+2
  int nq;       // Gauss points per element
  double h;     // element size
  double gq_t[TAPS_MAX_QUAD];  // Gauss abscissae on [0,1]
  double gq_w[TAPS_MAX_QUAD];  // Gauss weights on [0,1]
  cudaStream_t stream;
  double* d_ginv;       // [n][amax][pmax]: first |A| rows of each patch's G_i^{-1}
  double* d_N;          // [n-1][nq][nloc]
  double* d_B;          // [n-1][nq][nloc]
  double* d_xq;         // [n-1][nq]
  double* d_band_full;  // [TAPS_NUM_OPS][n][nb]
  double* d_band;       // [TAPS_NUM_OPS][nf][nb] restricted to the free nodes
  int* d_status;
  FdEntry fd[4];        // cached pencil decompositions
  int nfd;
};

// Term table passed by value to the kernels that combine dimensions.
struct TermTable {
  int D, R, Rf;
  double alpha[TAPS_MAX_TERMS];
  const double* beta;   // device array [Rf] (source amplitudes)
  signed char oi[TAPS_MAX_TERMS][TAPS_MAX_DIMS];  // distinct-op index of term t in dim d
  int nops[TAPS_MAX_DIMS];
  int cs;   // slot stride of the coefficient arrays: max(TAPS_NUM_OPS, max_d nops[d])
};

struct GramPtrs {
  const double* gram[TAPS_MAX_DIMS];  // [nops_d][M][M]
  const double* h[TAPS_MAX_DIMS];     // [Rf][M]
};

struct ProfPending {
  int cls;
  cudaEvent_t a, b;
};

struct ProfState {
  bool events;
  bool capturing;   // a sweep graph is being captured: record event nodes
  long long launches[TAPS_PROF_NUM];
  double ms[TAPS_PROF_NUM];
  double flops[TAPS_PROF_NUM];
  double bytes[TAPS_PROF_NUM];
  ProfPending pending[512];
  int npending;
  cudaEvent_t pool[1024];
  int npool;
};

struct taps_problem {
  int D, R, Rf;
  taps_dim* dims[TAPS_MAX_DIMS];
  cudaStream_t stream;
  TermTable tt;
  int ops[TAPS_MAX_DIMS][TAPS_MAX_SLOTS];  // op code of each distinct-op slot
  bool has_weighted;                       // some term uses a weighted operator
  unsigned long long wdef[TAPS_MAX_DIMS];  // weighted operators defined (bit j)
  unsigned long long wuse[TAPS_MAX_DIMS];  // weighted operators the terms use (bit j)
  double* d_wbuf;                          // nodal weights staged for assembly
  size_t wbuf_cap;
  int nf_max;
  double* d_q[TAPS_MAX_DIMS];            // [Rf][nf_d] source projections
  double* d_pq[TAPS_MAX_DIMS];           // [Rf][nf_d] Phi_d^T q_r (fast diagonalisation)
  double* d_beta;                        // [Rf] source amplitudes
  double* d_opband[TAPS_MAX_DIMS];       // [nops_d][nf_d][nb] bands of the distinct ops
  // Workspace, grown to the largest mode count seen (ws_M).
  int ws_M;
  double* d_gram[TAPS_MAX_DIMS];  // [nops_d][M][M]
  double* d_h[TAPS_MAX_DIMS];     // [Rf][M]
  double* d_C;        // [tt.cs][M][M] coefficient matrices of the current dim
  double* d_c;        // [Rf][M]
  double* d_Call;     // [D][tt.cs][M][M] coefficients of every dim (residual)
  double* d_call;     // [D][Rf][M]
  unsigned* d_ticket; // CTA tickets of the kernels whose last CTA finishes a reduction
  double* d_F;        // [nf_max][M] reduced right-hand side (node-major)
  double* d_blocks;   // [nf_max][nb][M][M] block band of the reduced matrix
  double* d_lu;       // [M][M] LU of the current diagonal block
  double* d_Y;        // [tt.cs][nf_max][M] SpMM products
  double* d_Uold;     // [nf_max][M]
  double* d_fdw;      // convection-face corrections: X [nf_max][2][M][M], w [nf_max][M], small parts
  double* d_md;       // mode-side solve: W [M][M], lam [M], W^T c [Rf][M], Z [nf_max][M],
                      // eliminated rows [nf_max][6][M]
  double* d_partial;  // partial sums of the Gram and residual kernels
  size_t partial_len;
  double* d_scal;     // small scalar scratch
  double* d_bigG;     // [D][NC][NC] residual Grams
  size_t bigG_len;
  double* d_Yres;     // [sum_d nops_d nf_d M] banded products of every dim (full residual)
  unsigned* d_ticket_all;   // [D][32] tickets of the all-dims Gram refresh
  int gram_all_ok;    // d_partial holds the chunk partials of every dim at once
  int* d_status;
  unsigned* d_bar;    // grid barrier words (count, generation)
  double* h_scal;     // pinned host mirror of d_scal
  double* h_part;     // pinned host mirror of the residual partial sums
  int* h_status;      // pinned host mirror of the device status word
  cudaStream_t cap_stream;  // private stream used to capture sweep graphs
  void* graph;        // cached sweep graph (SweepGraph, api.cu)
  void* loop_graph;   // cached device-side solve loop (LoopGraph, api.cu)
  double* d_Usnap[TAPS_MAX_DIMS];  // factor snapshot for the FP32 -> FP64 retry
  void* d_evalbuf;    // grow-only gathered rows of taps_eval_grid
  size_t evalbuf_len;
  int eval_attr_set;  // shared-memory opt-in of the reconstruction kernels done
  int lu_tuned[16][3];  // tuned block-elimination CTA counts: (n, M, CTAs)
  int n_lu_tuned;
  int coop_blocks;    // CTAs of the cooperative block solve
  // d_C / d_c hold dim 0's coefficients for the current Grams (the last dim's Gram
  // refresh of a sweep or of taps_refresh_grams forms them), so the next sweep need not
  int c0_valid;
  int c0_M;           // the mode count they were formed for (the layout of d_C)
  int c0_forbid;      // set around captures whose replays cannot rely on c0_valid
  int c0_skipped;     // a sweep enqueue reused them (read after a capture)
  int num_sms;
  ProfState* prof;
};

// Profiling helpers: prof_begin returns a token passed to prof_end.
int prof_begin(taps_problem* P, int cls);
void prof_end(taps_problem* P, int cls, int token, double flops, double bytes);
void prof_drain(taps_problem* P);

struct taps_factors {
  const taps_problem* prob;
  int M, M_cap;
  double* d_U[TAPS_MAX_DIMS];  // [nf_d][M_cap] column-major, leading dim nf_d
};

// ---------------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void taps_flag(int* status, int code) {
  atomicCAS(status, TAPS_DEV_OK, code);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Programmatic dependent launch.  A kernel launched by taps_launch_pdl may be
// scheduled while its predecessor on the stream is still running; it calls
// taps_pdl_wait() before its first global-memory access (the wait returns once the
// predecessor has completed and its writes are visible).  Launched without the
// attribute, the wait returns at once.  The kernels do not trigger their successor
// early (griddepcontrol.launch_dependents at their start): a successor released that
// way keeps all its CTAs resident and waiting beside the running kernel, which on this
// GPU stretched the node-side small solves from ~19 to ~60 us per launch on some dims
// (globaltimer traces of the whole sweep); released at exit, the successor's launch
// still overlaps the predecessor's tail.
__device__ __forceinline__ void taps_pdl_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t taps_launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                   cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg;
  memset(&cfg, 0, sizeof(cfg));
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

// FP64 reciprocal: the hardware's approximate reciprocal y0 refined by one step of
// the series 1/x = y0 / (1 - e) = y0 (1 + e + e^2 + ...), e = 1 - x y0 (the quadratic
// Newton-Raphson / series refinement of a reciprocal seed).  One approximate op and
// three dependent FMAs: within one ulp of 1.0 / x for normal x (the seed flushes
// subnormals), at about 60% of the IEEE division's dependent latency.
__device__ __forceinline__ double taps_rcp(double x) {
  double y0;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y0) : "d"(x));
  const double e = fma(-x, y0, 1.0);
  return fma(y0, fma(e, e, e), y0);
}

// A double that is neither zero nor infinite nor NaN, decided on its bits (integer
// operations: no FP64 compare, which would hold an FP64 pipe on this GPU ~64 cycles).
__device__ __forceinline__ bool taps_finite_nonzero(double x) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
  return u != 0ull && (u >> 52) != 0x7FFull;
}

// Block-wide sum for blockDim.x <= 1024; `red` holds >= 32 T in shared memory.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T* red) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? red[threadIdx.x] : T(0);
  if (w == 0) r = warp_sum(r);
  if (threadIdx.x == 0) red[0] = r;
  __syncthreads();
  r = red[0];
  __syncthreads();
  return r;
}

// Grid barrier for a cooperative launch (all CTAs co-resident).  Sense-reversal on
// a generation counter; every wait is bounded: after `limit` polls the barrier
// records TAPS_DEV_TIMEOUT and stops waiting, and later barriers return at once, so
// the kernel always runs to its end and the host reads the status.
__device__ __forceinline__ void grid_barrier(unsigned* bar, int* status, unsigned nblocks,
                                             long long limit = (1ll << 26)) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned* vgen = bar + 1;
    volatile int* vstat = status;
    if (*vstat != TAPS_DEV_TIMEOUT) {
      unsigned gen = *vgen;
      __threadfence();
      unsigned arrived = atomicAdd(bar, 1u);
      if (arrived == nblocks - 1) {
        atomicExch(bar, 0u);
        __threadfence();
        atomicAdd(bar + 1, 1u);
      } else {
        long long polls = 0;
        while (*vgen == gen) {
          if (++polls > limit) {  // default ~seconds: far above any legitimate wait
            taps_flag(status, TAPS_DEV_TIMEOUT);
            break;
          }
          if (*vstat == TAPS_DEV_TIMEOUT) break;
          __nanosleep(20);
        }
      }
      __threadfence();
    }
  }
  __syncthreads();
}

// SplitMix64 (Steele, Lea & Flood 2014): state += golden gamma, then the output mix.
__host__ __device__ __forceinline__ uint64_t splitmix64_mix(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Counter = seed (24 bits) | dim (8) | mode (12) | row (20); top 53 bits -> U(-1,1).
__host__ __device__ __forceinline__ double taps_uniform_pm1(unsigned seed, int d, int i, int m) {
  uint64_t ctr = ((uint64_t)(seed & 0xFFFFFFu) << 40) | ((uint64_t)(d & 0xFF) << 32) |
                 ((uint64_t)(m & 0xFFF) << 20) | (uint64_t)(i & 0xFFFFF);
  uint64_t z = splitmix64_mix(ctr);
  return 2.0 * ((double)(z >> 11) * (1.0 / 9007199254740992.0)) - 1.0;
}

// ---------------------------------------------------------------------------------
// Entry points between translation units
// ---------------------------------------------------------------------------------
int taps_ws_ensure(taps_problem* P, int M);
int taps_refresh_grams(taps_problem* P, const taps_factors* U, int precision);
// Coefficients of dim d from the current Grams into P->d_C / P->d_c.
int taps_coefficients(taps_problem* P, int d, int M);
// Largest dynamic shared memory a launch of `fn` may ask for (opt-in limit less the
// kernel's static shared memory).
int taps_allow_dyn_smem(const void* fn, int maxsm);

// Grid of a reconstruction: per dim the number of nodes and the offset of its
// gathered factor rows [count][M].
struct GridSpec {
  int D;
  int count[TAPS_MAX_DIMS];
  long long goff[TAPS_MAX_DIMS];
};
// Tensor-core reconstruction of an FP32 grid (rank-M product of the leading dims'
// and the trailing dims' row products).
int taps_eval_tc_usable(long long rows, long long cols, int M);
size_t taps_eval_tc_scratch(long long rows, long long cols, int M);
int taps_eval_tc_setup(int maxsm);
int taps_eval_tc(taps_problem* P, const float* G, const GridSpec& gs, int split, int M, long long rows,
                 long long cols, void* scratch, float* out);
// Gram refresh of dim d; with coeff_dim >= 0 the same launch then forms the
// coefficients of dim coeff_dim in P->d_C / P->d_c.
int taps_refresh_gram_dim(taps_problem* P, const taps_factors* U, int d, int precision,
                          int coeff_dim);
int taps_sweep_impl(taps_problem* P, taps_factors* U, int precision, int solver, int normalize,
                    double* change_out);
int taps_residual_impl(taps_problem* P, const taps_factors* U, int kind, double* rho_out,
                       int grams_current = 0);
// host_copies = 0 leaves the change partials and the status word on the device (the
// device-side solve loop reads them there).
int taps_sweep_enqueue(taps_problem* P, taps_factors* U, int precision, int solver, int normalize,
                       int host_copies = 1);
int taps_sweep_finish(taps_problem* P, taps_factors* U, double* change_out);
// After a sweep and/or a residual enqueued without host copies: nscal change partials,
// npart residual partials and the status word into the pinned host buffers that the
// finish functions read.
int taps_results_to_host(taps_problem* P, int nscal, int npart);
// Number of partial sums a residual of this kind leaves in P->d_partial.
int taps_residual_npart(const taps_problem* P, int kind);
// grams_current: the FP64 Grams and source projections of every dim already belong to
// U (true right after an FP64 or MIXED sweep), so the ALS residual does not refresh them.
int taps_residual_enqueue(taps_problem* P, const taps_factors* U, int kind, int grams_current = 0,
                          int host_copies = 1);
// Per-dim ranges of the ALS residual's partial sums (CTA indices [cta0[d], cta0[d+1])).
int taps_als_partial_ranges(const taps_problem* P, int* cta0);
int taps_residual_finish(taps_problem* P, const taps_factors* U, int kind, double* rho_out);
// Reduced-precision Gram contractions (FP32 or BF16-rounded inputs, FP32 accumulation).
static inline bool taps_low_prec(int precision) { return precision == TAPS_FP32 || precision == TAPS_BF16; }

// How dim d is solved at M modes under `solver`.
#define TAPS_ROUTE_LU 0
#define TAPS_ROUTE_FD 1   // node-side pencil (fastdiag.cu)
#define TAPS_ROUTE_MD 2   // mode-side pencil (modediag.cu)
#define TAPS_ROUTE_FDW 3  // node-side pencil with convection-face corrections (fdbound.cu)
int taps_dim_route(const taps_problem* P, int d, int solver, int M);
int taps_fd_prepare_all(taps_problem* P, int solver, int M);
// Temporaries of one pencil decomposition in flight (fastdiag.cu).
struct FdPending {
  FdEntry* E;
  taps_problem* P;
  double *A, *B, *V, *tmp, *bt, *dd, *ee, *lam, *W;
};
// Mode-side diagonalisation (modediag.cu): eligibility of dim d at M modes (slots of
// the mass-like operator X and the other Y), scratch size, and the solve.
int taps_md_eligible(const taps_problem* P, int d, int M, int* slotX, int* slotY);
size_t taps_md_scratch_doubles(int nf_max, int M, int Rf);
int taps_md_setup(int maxsm);

// Tensor-core (tcgen05, BF16 operands, FP32 accumulation) Gram refresh (gram_tc.cu).
int taps_gram_tc_eligible(int M, int nops, int Rf, int hb);
int taps_gram_tc_setup(int maxsm);
int taps_gram_tc_single(const double* U, const double* band, const double* q, double* gram, double* h, int n,
                        int M, int hb, int nops, int Rf, double* partial, unsigned* ticket, int rows,
                        cudaStream_t s, int* status);
struct GtHostItem {
  const double *U, *band, *q;
  double *gram, *h;
  int n, M, hb, nops, Rf;
};
size_t taps_gram_tc_queue_bytes(int nitems, int max_tasks);
int taps_gram_tc_queue(const std::vector<GtHostItem>& hitems, int rows, int cpt, int ctas, void* dev_buf,
                       size_t dev_buf_bytes, double* partial, size_t partial_doubles, unsigned* tickets,
                       cudaStream_t s, int* status, double* flops_out, double* bytes_out, cudaEvent_t ev0,
                       cudaEvent_t ev1);
int taps_gram_tc_footprint(int rows, int maxN, int maxNH, int maxops, size_t* smem, int* ncols);
int taps_md_solve(taps_problem* P, taps_factors* U, int d);
int taps_md_reset(taps_problem* P);
// Node-side diagonalisation with convection-face corrections (fdbound.cu).
int taps_fdw_eligible(const taps_problem* P, int d, int M, int* slotA, int* slotB, int* slotC0, int* slotC1,
                      int* nbnd);
size_t taps_fdw_scratch_doubles(int nf_max, int M);
int taps_fdw_solve(taps_problem* P, taps_factors* U, int d);
int taps_fd_lookup(taps_problem* P, int d, int opA, int opB, const FdEntry** out);
int taps_fd_to_nodal(taps_problem* P, const FdEntry* E, const double* Y, int n, int M, double* Out, double* Save);
int taps_fd_prepare_enqueue(taps_problem* P, int solver, int M, std::vector<FdPending>* pend);
int taps_fd_prepare_finish(std::vector<FdPending>* pend);
int taps_lu_needs_tuning(const taps_problem* P, int solver, int M);
int taps_check_status(int* d_status, cudaStream_t s);
int taps_fd_eligible(const taps_problem* P, int d, int* slotA, int* slotB);
int taps_fd_solve(taps_problem* P, taps_factors* U, int d, int precision);
void taps_fd_release(taps_dim* dm);
