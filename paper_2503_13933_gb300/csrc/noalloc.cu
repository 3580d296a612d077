// Allocation-free grid reconstruction: taps_eval_grid_noalloc.
//
// Some callers cannot allocate device memory at the moment they need a field: code
// running while another component owns a fixed memory budget (a pre-sized pool with
// no headroom), code called back from inside a framework that forbids allocation on
// its hot path, or code that must not trigger the implicit synchronisation an
// allocation can cause.  This entry point computes the same values as
// taps_eval_grid but takes its working memory from one fixed array in device global
// memory that the library reserves when it is loaded.
#include "taps_internal.cuh"

// Fixed scratch: the gathered factor rows, sum_d count[d] * M values of the output
// type.  Every GPU that loads the library holds these bytes until the process exits.
static __device__ __align__(256) unsigned char taps_noalloc_scratch[TAPS_NOALLOC_SCRATCH_BYTES];

// Host code must not pass `taps_noalloc_scratch` itself to a kernel: in host code
// that name is a host-side shadow, not a device address.  The device address is looked
// up on every call, with the calling device current: the lookup allocates nothing and
// costs far less than the launches, and a cached address could go stale once the
// device's primary context is reset (cudaDeviceReset) or the module is reloaded.  The
// first lookup on a device may load the library's device code into the context, which
// is why the first call on a device should come before any stream capture.
static int noalloc_scratch_address(void** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, taps_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    taps_note_cuda_error(e, "cudaGetSymbolAddress(taps_noalloc_scratch)", __FILE__, __LINE__);
    return TAPS_ERR_CUDA;
  }
  *out = p;
  return TAPS_OK;
}

struct NoallocGrid {
  int D;
  int count[TAPS_MAX_DIMS];
  int goff[TAPS_MAX_DIMS];
};

template <typename T>
__global__ void noalloc_gather_kernel(const double* U, int nf, int off, int start, int step, int count,
                                      int M, T* G) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= count * M) return;
  int j = idx / M, m = idx - j * M;
  int fj = start + step * j - off;
  G[idx] = (fj >= 0 && fj < nf) ? (T)U[(size_t)m * nf + fj] : (T)0;
}

// A CTA owns NR consecutive rows of the leading dims (all dims but the last) and all
// entries of the last dim: the rows' factor products are formed in shared memory,
// then every output is one length-M dot product against a last-dim factor row.
#define NR 8
static_assert(NR * TAPS_MAX_M * sizeof(double) <= 48 * 1024, "noalloc eval rows exceed the default shared memory");
template <typename T>
__global__ void __launch_bounds__(256) noalloc_eval_kernel(const T* __restrict__ G, NoallocGrid g, int M,
                                                           long long rows, T* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char sm[];
  T* Pr = reinterpret_cast<T*>(sm);  // [NR][M]
  const int last = g.count[g.D - 1];
  const long long r0 = (long long)blockIdx.x * NR;
  const int nr = (int)min((long long)NR, rows - r0);
  for (int idx = threadIdx.x; idx < nr * M; idx += blockDim.x) {
    int rr = idx / M, m = idx - rr * M;
    long long row = r0 + rr;
    T v = (T)1;
    for (int d = g.D - 2; d >= 0; --d) {
      long long q = row / g.count[d];
      int id = (int)(row - q * g.count[d]);
      row = q;
      v *= G[g.goff[d] + id * M + m];
    }
    Pr[rr * M + m] = v;
  }
  __syncthreads();
  const T* GL = G + g.goff[g.D - 1];
  const int nout = nr * last;
  for (int o = threadIdx.x; o < nout; o += blockDim.x) {
    int rr = o / last, j = o - rr * last;
    const T* p = Pr + rr * M;
    const T* gl = GL + j * M;
    T acc = (T)0;
    for (int m = 0; m < M; ++m) acc += p[m] * gl[m];
    out[(r0 + rr) * last + j] = acc;
  }
}

extern "C" int taps_eval_grid_noalloc(const taps_problem* P, const taps_factors* U, const int* start,
                                      const int* count, const int* step, void* out_dev, int out_dtype) {
  if (!P || !U || !start || !count || !step || !out_dev || U->M < 1) return TAPS_ERR_INVALID_ARG;
  if (out_dtype != TAPS_FP64 && out_dtype != TAPS_FP32) return TAPS_ERR_INVALID_ARG;
  const int M = U->M;
  const size_t esz = out_dtype == TAPS_FP64 ? sizeof(double) : sizeof(float);
  NoallocGrid g;
  g.D = P->D;
  long long total = 1, goff = 0;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    if (count[d] < 1) return TAPS_ERR_INVALID_ARG;
    long long first = start[d], lastn = start[d] + (long long)step[d] * (count[d] - 1);
    if (first < 0 || first >= dm->n || lastn < 0 || lastn >= dm->n) return TAPS_ERR_INVALID_ARG;
    g.count[d] = count[d];
    g.goff[d] = (int)goff;
    goff += (long long)count[d] * M;
    total *= count[d];
  }
  if ((size_t)goff * esz > (size_t)TAPS_NOALLOC_SCRATCH_BYTES) return TAPS_ERR_SCRATCH_LIMIT;
  // the eval kernel's shared rows: at most NR * TAPS_MAX_M doubles (8 KB), inside the
  // 48 KB every launch may use without an opt-in; checked before anything is launched
  const size_t smem = (size_t)NR * M * esz;
  if (M > TAPS_MAX_M || smem > 48u * 1024u) return TAPS_ERR_INVALID_ARG;
  void* scratch = nullptr;
  TAPS_TRY(noalloc_scratch_address(&scratch));
  cudaStream_t s = P->stream;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    int n = count[d] * M;
    if (out_dtype == TAPS_FP64)
      noalloc_gather_kernel<double><<<(n + 255) / 256, 256, 0, s>>>(
          U->d_U[d], dm->nf, dm->off, start[d], step[d], count[d], M, (double*)scratch + g.goff[d]);
    else
      noalloc_gather_kernel<float><<<(n + 255) / 256, 256, 0, s>>>(
          U->d_U[d], dm->nf, dm->off, start[d], step[d], count[d], M, (float*)scratch + g.goff[d]);
    TAPS_CUDA(cudaGetLastError());
  }
  long long rows = total / count[P->D - 1];
  unsigned blocks = (unsigned)((rows + NR - 1) / NR);
  if (out_dtype == TAPS_FP64)
    noalloc_eval_kernel<double><<<blocks, 256, smem, s>>>((const double*)scratch, g, M, rows, (double*)out_dev);
  else
    noalloc_eval_kernel<float><<<blocks, 256, smem, s>>>((const float*)scratch, g, M, rows, (float*)out_dev);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}
