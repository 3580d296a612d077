// 1D C-HiDeNN assembly on the device: patch inverses (Eq. 1), shape-function tables
// at the Gauss points (Table 1), banded K, M, G, W, B matrices (Eqs. 31-35) and
// source projections (forcing term of Eq. 30).
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "taps_internal.cuh"

// ---------------------------------------------------------------------------------
// Status, errors, allocation
// ---------------------------------------------------------------------------------
static char g_last_cuda[256];

void taps_note_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
  snprintf(g_last_cuda, sizeof(g_last_cuda), "%s:%d %s: %s", file, line, what,
           cudaGetErrorString(e));
  if (getenv("TAPS_VERBOSE")) fprintf(stderr, "[taps] %s\n", g_last_cuda);
}

int taps_alloc(void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    return TAPS_ERR_OOM;
  }
  TAPS_CUDA(e);
  return TAPS_OK;
}

int taps_status_from_device(int dev) {
  switch (dev) {
    case TAPS_DEV_OK: return TAPS_OK;
    case TAPS_DEV_SINGULAR: return TAPS_ERR_SINGULAR;
    case TAPS_DEV_NONFINITE: return TAPS_ERR_NONFINITE;
    case TAPS_DEV_TIMEOUT: return TAPS_ERR_TIMEOUT;
    default: return TAPS_ERR_CUDA;
  }
}

// Read and clear a device status word (synchronises the stream).
int taps_check_status(int* d_status, cudaStream_t s) {
  int h = 0;
  TAPS_CUDA(cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  TAPS_CUDA(cudaStreamSynchronize(s));
  if (h != TAPS_DEV_OK) {
    TAPS_CUDA(cudaMemsetAsync(d_status, 0, sizeof(int), s));
    TAPS_CUDA(cudaStreamSynchronize(s));
  }
  return taps_status_from_device(h);
}

extern "C" const char* taps_status_string(int status) {
  switch (status) {
    case TAPS_OK: return "ok";
    case TAPS_ERR_INVALID_ARG: return "invalid argument";
    case TAPS_ERR_SINGULAR: return "singular pivot";
    case TAPS_ERR_NONFINITE: return "non-finite value";
    case TAPS_ERR_NOT_CONVERGED: return "not converged";
    case TAPS_ERR_TIMEOUT: return "device wait timed out";
    case TAPS_ERR_CUDA: return g_last_cuda[0] ? g_last_cuda : "CUDA error";
    case TAPS_ERR_OOM: return "out of device memory";
    case TAPS_ERR_SCRATCH_LIMIT:
      return "request exceeds the fixed scratch of taps_eval_grid_noalloc (TAPS_NOALLOC_SCRATCH_BYTES)";
    default: return "unknown status";
  }
}

extern "C" int taps_version(void) { return 1; }

// ---------------------------------------------------------------------------------
// Gauss-Legendre rule on [0, 1]: Newton iteration on the Legendre recurrence.
// ---------------------------------------------------------------------------------
static void gauss_legendre01(int nq, double* t, double* w) {
  std::vector<std::pair<double, double>> pw;
  for (int i = 0; i < nq; ++i) {
    double x = cos(M_PI * (i + 0.75) / (nq + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= nq; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (nq == 1) { p0 = 1.0; p1 = x; }
      dp = nq * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    {  // derivative at the converged root
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= nq; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (nq == 1) p0 = 1.0;
      dp = nq * (x * p1 - p0) / (x * x - 1.0);
    }
    pw.push_back({x, 2.0 / ((1.0 - x * x) * dp * dp)});
  }
  std::sort(pw.begin(), pw.end());
  for (int i = 0; i < nq; ++i) {
    t[i] = 0.5 * (pw[i].first + 1.0);
    w[i] = 0.5 * pw[i].second;
  }
}

// ---------------------------------------------------------------------------------
// Kernels
// ---------------------------------------------------------------------------------
struct DimParams {
  int n, s, p, nq, amax, pmax, nloc, hb, nb, nf, off;
  double a, lo, hi, step;
  double gq_t[TAPS_MAX_QUAD], gq_w[TAPS_MAX_QUAD];
  double wpoly[4];
};

__device__ __forceinline__ double node_x(const DimParams& P, int j) {
  return (j == P.n - 1) ? P.hi : P.lo + j * P.step;
}

// Cubic-spline window of the patch function (support |z| <= 1).
__device__ __forceinline__ double spline_phi(double z) {
  z = fabs(z);
  if (z <= 0.5) return 2.0 / 3.0 - 4.0 * z * z + 4.0 * z * z * z;
  if (z <= 1.0) return 4.0 / 3.0 - 4.0 * z + 4.0 * z * z - 4.0 / 3.0 * z * z * z;
  return 0.0;
}
__device__ __forceinline__ double spline_dphi(double z) {
  z = fabs(z);
  if (z <= 0.5) return -8.0 * z + 12.0 * z * z;
  if (z <= 1.0) return -4.0 + 8.0 * z - 4.0 * z * z;
  return 0.0;
}

#define PMAXC (2 * TAPS_MAX_S + 1 + TAPS_MAX_P + 1)

// One thread per node i: invert the moment matrix G_i = [[R, P], [P^T, 0]] of the
// node's convolution patch (Gauss-Jordan, partial pivoting) and keep the rows of the
// patch nodes.  The patch function is then W^i(x) = G_i^{-1}[rows] [phi(x); P(x)].
__global__ void patch_inverse_kernel(DimParams P, double* ginv, int* status) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.n) return;
  double h = P.step;
  int j0 = max(0, i - P.s), j1 = min(P.n - 1, i + P.s);
  int na = j1 - j0 + 1, np = na + P.p + 1;
  double G[PMAXC][2 * PMAXC];
  for (int r = 0; r < np; ++r)
    for (int c = 0; c < 2 * np; ++c) G[r][c] = 0.0;
  double xi = node_x(P, i);
  for (int r = 0; r < na; ++r) {
    double xr = node_x(P, j0 + r);
    for (int c = 0; c < na; ++c) G[r][c] = spline_phi(fabs(xr - node_x(P, j0 + c)) / (P.a * h));
    double t = (xr - xi) / h, pw = 1.0;
    for (int q = 0; q <= P.p; ++q) {
      G[r][na + q] = pw;
      G[na + q][r] = pw;
      pw *= t;
    }
  }
  for (int r = 0; r < np; ++r) G[r][np + r] = 1.0;
  for (int c = 0; c < np; ++c) {
    int piv = c;
    double best = fabs(G[c][c]);
    for (int r = c + 1; r < np; ++r)
      if (fabs(G[r][c]) > best) { best = fabs(G[r][c]); piv = r; }
    if (!(best > 0.0) || !isfinite(best)) {
      taps_flag(status, TAPS_DEV_SINGULAR);
      return;
    }
    if (piv != c)
      for (int k = 0; k < 2 * np; ++k) { double tmp = G[c][k]; G[c][k] = G[piv][k]; G[piv][k] = tmp; }
    double inv = 1.0 / G[c][c];
    for (int k = 0; k < 2 * np; ++k) G[c][k] *= inv;
    for (int r = 0; r < np; ++r) {
      if (r == c) continue;
      double f = G[r][c];
      if (f != 0.0)
        for (int k = 0; k < 2 * np; ++k) G[r][k] -= f * G[c][k];
    }
  }
  double* out = ginv + (size_t)i * P.amax * P.pmax;
  for (int r = 0; r < P.amax; ++r)
    for (int l = 0; l < P.pmax; ++l)
      out[r * P.pmax + l] = (r < na && l < np) ? G[r][np + l] : 0.0;
}

// One thread per (element e, Gauss point g): C-HiDeNN shape functions and their
// derivatives N~_k = N_e W^e_k + N_{e+1} W^{e+1}_k for the 2s+2 nodes of the element.
__global__ void shape_kernel(DimParams P, const double* ginv, double* Nt, double* Bt, double* xq) {
  int e = blockIdx.x;
  int g = threadIdx.x;
  if (e >= P.n - 1 || g >= P.nq) return;
  double xe0 = node_x(P, e), xe1 = node_x(P, e + 1);
  double he = xe1 - xe0;
  double x = xe0 + P.gq_t[g] * he;
  double N[2 * TAPS_MAX_S + 2], B[2 * TAPS_MAX_S + 2];
  for (int k = 0; k < P.nloc; ++k) { N[k] = 0.0; B[k] = 0.0; }
  double hat[2] = {(xe1 - x) / he, (x - xe0) / he};
  double dhat[2] = {-1.0 / he, 1.0 / he};
  double h = P.step;
  for (int c = 0; c < 2; ++c) {
    int i = e + c;
    int j0 = max(0, i - P.s), j1 = min(P.n - 1, i + P.s);
    int na = j1 - j0 + 1, np = na + P.p + 1;
    double row[PMAXC], drow[PMAXC];
    for (int r = 0; r < na; ++r) {
      double d = x - node_x(P, j0 + r);
      double z = fabs(d) / (P.a * h);
      row[r] = spline_phi(z);
      drow[r] = spline_dphi(z) * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (P.a * h);
    }
    double t = (x - node_x(P, i)) / h, pw = 1.0, dpw = 0.0;
    for (int q = 0; q <= P.p; ++q) {
      row[na + q] = pw;
      drow[na + q] = dpw / h;
      dpw = (q + 1) * pw;  // d/dt t^{q+1} = (q+1) t^q
      pw *= t;
    }
    const double* Gi = ginv + (size_t)i * P.amax * P.pmax;
    for (int r = 0; r < na; ++r) {
      double W = 0.0, dW = 0.0;
      for (int l = 0; l < np; ++l) {
        W += Gi[r * P.pmax + l] * row[l];
        dW += Gi[r * P.pmax + l] * drow[l];
      }
      int k = (j0 + r) - (e - P.s);
      N[k] += hat[c] * W;
      B[k] += dhat[c] * W + hat[c] * dW;
    }
  }
  size_t base = ((size_t)e * P.nq + g) * P.nloc;
  for (int k = 0; k < P.nloc; ++k) { Nt[base + k] = N[k]; Bt[base + k] = B[k]; }
  xq[(size_t)e * P.nq + g] = x;
}

// One thread per (op; node i; band offset k): for K, M, G, W element-by-element Gauss
// sums of Eqs. 33-35 over the elements shared by nodes i and j = i + k - hb; for Blo,
// Bhi the point mass at the end node (a face integral through the Kronecker delta).
__global__ void band_kernel(DimParams P, const double* Nt, const double* Bt, const double* xq,
                            double* band_full) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)TAPS_NUM_OPS * P.n * P.nb;
  if (idx >= total) return;
  int k = idx % P.nb;
  int i = (idx / P.nb) % P.n;
  int op = idx / ((long long)P.nb * P.n);
  int j = i + k - P.hb;
  double v = 0.0;
  if (op == TAPS_OP_BLO || op == TAPS_OP_BHI) {
    const int end = op == TAPS_OP_BLO ? 0 : P.n - 1;
    band_full[idx] = (i == end && j == end) ? 1.0 : 0.0;
    return;
  }
  if (j >= 0 && j < P.n) {
    int e_lo = max(max(i, j) - P.s - 1, 0);
    int e_hi = min(min(i, j) + P.s, P.n - 2);
    for (int e = e_lo; e <= e_hi; ++e) {
      double he = node_x(P, e + 1) - node_x(P, e);
      int li = i - (e - P.s), lj = j - (e - P.s);
      for (int g = 0; g < P.nq; ++g) {
        size_t base = ((size_t)e * P.nq + g) * P.nloc;
        double wj = P.gq_w[g] * he;
        double term;
        if (op == TAPS_OP_K) term = Bt[base + li] * Bt[base + lj];
        else if (op == TAPS_OP_M) term = Nt[base + li] * Nt[base + lj];
        else if (op == TAPS_OP_G) term = Nt[base + li] * Bt[base + lj];
        else {
          double x = xq[(size_t)e * P.nq + g];
          double w = P.wpoly[0] + P.wpoly[1] * x + P.wpoly[2] * x * x + P.wpoly[3] * x * x * x;
          term = w * Nt[base + li] * Nt[base + lj];
        }
        v += wj * term;
      }
    }
  }
  band_full[((size_t)op * P.n + i) * P.nb + k] = v;
}

// Weighted operator over the free nodes (App. A): one thread per (free row fi, band
// offset k), Gauss sums over the elements shared by nodes i and j = i + k - hb of
//   K: w B~_i B~_j,   M: w N~_i N~_j,   G: N~_i (w' N~_j + w B~_j),
// with w and w' the C-HiDeNN interpolant of the nodal weights (all nodes) and its
// derivative at the Gauss point, summed over the element's patch nodes.  Entries
// whose column is a constrained node are 0 (the restriction of restrict_kernel).
// Every weighted operator of one dim in one launch: blockIdx.y = operator, its base,
// weight row and output band from the table.
struct WeightedOps {
  int count;
  int base[TAPS_MAX_SLOTS];
  int wrow[TAPS_MAX_SLOTS];   // row of the weights array
  int slot[TAPS_MAX_SLOTS];   // band slot in the output
};

__global__ void weighted_band_kernel(DimParams P, const double* Nt, const double* Bt, WeightedOps ops,
                                     const double* __restrict__ wall, double* __restrict__ bands) {
  const int o = blockIdx.y;
  const int base = ops.base[o];
  const double* __restrict__ w = wall + (size_t)ops.wrow[o] * P.n;
  double* __restrict__ band = bands + (size_t)ops.slot[o] * P.nf * P.nb;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)P.nf * P.nb) return;
  const int k = (int)(idx % P.nb);
  const int fi = (int)(idx / P.nb);
  const int i = fi + P.off, j = i + k - P.hb;
  double v = 0.0;
  if (j >= P.off && j < P.off + P.nf) {
    const int e_lo = max(max(i, j) - P.s - 1, 0);
    const int e_hi = min(min(i, j) + P.s, P.n - 2);
    for (int e = e_lo; e <= e_hi; ++e) {
      const double he = node_x(P, e + 1) - node_x(P, e);
      const int li = i - (e - P.s), lj = j - (e - P.s);
      for (int g = 0; g < P.nq; ++g) {
        const size_t base_idx = ((size_t)e * P.nq + g) * P.nloc;
        double wv = 0.0, dw = 0.0;
        for (int l = 0; l < P.nloc; ++l) {
          const int node = e - P.s + l;
          if (node >= 0 && node < P.n) {
            wv += Nt[base_idx + l] * w[node];
            dw += Bt[base_idx + l] * w[node];
          }
        }
        double term;
        if (base == TAPS_OP_K) term = wv * Bt[base_idx + li] * Bt[base_idx + lj];
        else if (base == TAPS_OP_M) term = wv * Nt[base_idx + li] * Nt[base_idx + lj];
        else term = Nt[base_idx + li] * (dw * Nt[base_idx + lj] + wv * Bt[base_idx + lj]);
        v += P.gq_w[g] * he * term;
      }
    }
  }
  band[idx] = v;
}

// Restriction of every band to the free nodes.
__global__ void restrict_kernel(DimParams P, const double* band_full, double* band) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)TAPS_NUM_OPS * P.nf * P.nb;
  if (idx >= total) return;
  int k = idx % P.nb;
  int fi = (idx / P.nb) % P.nf;
  int op = idx / ((long long)P.nb * P.nf);
  int i = fi + P.off, j = i + k - P.hb;
  double v = band_full[((size_t)op * P.n + i) * P.nb + k];
  bool jfree = (j >= P.off) && (j < P.off + P.nf);
  band[idx] = jfree ? v : 0.0;
}

__device__ __forceinline__ double source_factor(int kind, const double* par, double x) {
  switch (kind) {
    case TAPS_SRC_CONST: return par[0];
    case TAPS_SRC_SIN: return sin(par[0] * x + par[1]);
    case TAPS_SRC_GAUSS: {
      double d = x - par[0];
      return exp(-(d * d) / (2.0 * par[1] * par[1]));
    }
    case TAPS_SRC_POLY: return par[0] + par[1] * x + par[2] * x * x + par[3] * x * x * x;
    default: return 0.0;
  }
}

// q_i = int N~_i g (Gauss sums over the elements touching node i), or for nodal
// data q = M_full g; written for the free nodes only.
__device__ __forceinline__ void source_entry(const DimParams& P, const double* Nt, const double* xq,
                                             const double* band_full, const double* band_free, int kind,
                                             double p0, double p1, double p2, double p3, const double* nodal,
                                             double* q_free, int fi) {
  int i = fi + P.off;
  double par[4] = {p0, p1, p2, p3};
  double v = 0.0;
  if (kind == TAPS_SRC_OPVEC_FULL) {   // q = (Op v)[free] for v at all nodes
    const double* row = band_full + ((size_t)(int)p0 * P.n + i) * P.nb;
    for (int k = 0; k < P.nb; ++k) {
      int j = i + k - P.hb;
      if (j >= 0 && j < P.n) v += row[k] * nodal[j];
    }
  } else if (kind == TAPS_SRC_OPVEC) {   // q = Op v on the free nodes
    const double* row = band_free + ((size_t)(int)p0 * P.nf + fi) * P.nb;
    for (int k = 0; k < P.nb; ++k) {
      int fj = fi + k - P.hb;
      if (fj >= 0 && fj < P.nf) v += row[k] * nodal[fj];
    }
  } else if (kind == TAPS_SRC_NODAL) {
    const double* Mrow = band_full + ((size_t)TAPS_OP_M * P.n + i) * P.nb;
    for (int k = 0; k < P.nb; ++k) {
      int j = i + k - P.hb;
      if (j >= 0 && j < P.n) v += Mrow[k] * nodal[j];
    }
  } else {
    int e_lo = max(i - P.s - 1, 0), e_hi = min(i + P.s, P.n - 2);
    for (int e = e_lo; e <= e_hi; ++e) {
      double he = node_x(P, e + 1) - node_x(P, e);
      int li = i - (e - P.s);
      for (int g = 0; g < P.nq; ++g) {
        double x = xq[(size_t)e * P.nq + g];
        v += P.gq_w[g] * he * source_factor(kind, par, x) * Nt[((size_t)e * P.nq + g) * P.nloc + li];
      }
    }
  }
  q_free[fi] = v;
}

__global__ void source_kernel(DimParams P, const double* Nt, const double* xq,
                              const double* band_full, const double* band_free, int kind, double p0,
                              double p1, double p2, double p3, const double* nodal, double* q_free) {
  int fi = blockIdx.x * blockDim.x + threadIdx.x;
  if (fi >= P.nf) return;
  source_entry(P, Nt, xq, band_full, band_free, kind, p0, p1, p2, p3, nodal, q_free, fi);
}

// Every source factor of one dim at once (blockIdx.y = source r): the same entry
// arithmetic as source_kernel; kinds, parameters and the offsets of the nodal data in
// one packed device buffer.
__global__ void source_all_kernel(DimParams P, const double* Nt, const double* xq, const double* band_full,
                                  const double* band_free, const int* kinds, const double* pars,
                                  const long long* offs, const double* nodal, double* q) {
  const int fi = blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (fi >= P.nf) return;
  const double* pr = pars + 4 * (size_t)r;
  source_entry(P, Nt, xq, band_full, band_free, kinds[r], pr[0], pr[1], pr[2], pr[3],
               offs[r] >= 0 ? nodal + offs[r] : nullptr, q + (size_t)r * P.nf, fi);
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
static DimParams make_params(const taps_dim* d) {
  DimParams P;
  memset(&P, 0, sizeof(P));
  P.n = d->n;
  P.s = d->desc.s;
  P.p = d->desc.p;
  P.nq = d->nq;
  P.amax = d->amax;
  P.pmax = d->pmax;
  P.nloc = d->nloc;
  P.hb = d->hb;
  P.nb = d->nb;
  P.nf = d->nf;
  P.off = d->off;
  P.a = d->desc.a;
  P.lo = d->desc.lo;
  P.hi = d->desc.hi;
  P.step = d->h;
  for (int g = 0; g < d->nq; ++g) { P.gq_t[g] = d->gq_t[g]; P.gq_w[g] = d->gq_w[g]; }
  for (int c = 0; c < 4; ++c) P.wpoly[c] = d->desc.weight_poly[c];
  return P;
}

extern "C" void taps_dim_destroy(taps_dim* d) {
  if (!d) return;
  if (d->stream) cudaStreamSynchronize(d->stream);
  taps_fd_release(d);
  cudaFree(d->d_ginv);
  cudaFree(d->d_N);
  cudaFree(d->d_B);
  cudaFree(d->d_xq);
  cudaFree(d->d_band_full);
  cudaFree(d->d_band);
  cudaFree(d->d_status);
  delete d;
}

static int assemble_impl(taps_dim* d) {
  DimParams P = make_params(d);
  cudaStream_t s = d->stream;
  int n = d->n;
  TAPS_TRY(taps_alloc((void**)&d->d_status, sizeof(int)));
  TAPS_CUDA(cudaMemsetAsync(d->d_status, 0, sizeof(int), s));
  TAPS_TRY(taps_alloc((void**)&d->d_ginv, sizeof(double) * n * d->amax * d->pmax));
  TAPS_TRY(taps_alloc((void**)&d->d_N, sizeof(double) * (n - 1) * d->nq * d->nloc));
  TAPS_TRY(taps_alloc((void**)&d->d_B, sizeof(double) * (n - 1) * d->nq * d->nloc));
  TAPS_TRY(taps_alloc((void**)&d->d_xq, sizeof(double) * (n - 1) * d->nq));
  TAPS_TRY(taps_alloc((void**)&d->d_band_full, sizeof(double) * TAPS_NUM_OPS * n * d->nb));
  TAPS_TRY(taps_alloc((void**)&d->d_band, sizeof(double) * TAPS_NUM_OPS * d->nf * d->nb));
  TAPS_CUDA(cudaMemsetAsync(d->d_band_full, 0, sizeof(double) * TAPS_NUM_OPS * n * d->nb, s));
  patch_inverse_kernel<<<(n + 63) / 64, 64, 0, s>>>(P, d->d_ginv, d->d_status);
  TAPS_CUDA(cudaGetLastError());
  shape_kernel<<<n - 1, 32, 0, s>>>(P, d->d_ginv, d->d_N, d->d_B, d->d_xq);
  TAPS_CUDA(cudaGetLastError());
  long long tot = (long long)TAPS_NUM_OPS * n * d->nb;
  band_kernel<<<(unsigned)((tot + 127) / 128), 128, 0, s>>>(P, d->d_N, d->d_B, d->d_xq,
                                                            d->d_band_full);
  TAPS_CUDA(cudaGetLastError());
  long long tr = (long long)TAPS_NUM_OPS * d->nf * d->nb;
  restrict_kernel<<<(unsigned)((tr + 127) / 128), 128, 0, s>>>(P, d->d_band_full, d->d_band);
  TAPS_CUDA(cudaGetLastError());
  return taps_check_status(d->d_status, s);
}

extern "C" int taps_assemble_1d(const taps_dim_desc* desc, void* stream, taps_dim** out) {
  if (!desc || !out) return TAPS_ERR_INVALID_ARG;
  *out = nullptr;
  const taps_dim_desc& D = *desc;
  if (D.n < 2 || D.s < 0 || D.s > TAPS_MAX_S || D.p < 0 || D.p > TAPS_MAX_P ||
      D.n_quad < 1 || D.n_quad > TAPS_MAX_QUAD || !(D.hi > D.lo) || !(D.a > 0.0) ||
      D.kind < TAPS_SPACE || D.kind > TAPS_TIME)
    return TAPS_ERR_INVALID_ARG;
  // Truncated end patches must hold p+1 nodes to reproduce order p.
  if (std::min(D.s, D.n - 1) + 1 < D.p + 1) return TAPS_ERR_INVALID_ARG;
  int nf = D.n - (D.dirichlet_lo ? 1 : 0) - (D.dirichlet_hi ? 1 : 0);
  if (nf < 1) return TAPS_ERR_INVALID_ARG;
  taps_dim* d = new taps_dim();
  memset((void*)d, 0, sizeof(taps_dim));
  d->desc = D;
  d->n = D.n;
  d->nf = nf;
  d->off = D.dirichlet_lo ? 1 : 0;
  d->hb = 2 * D.s + 1;
  d->nb = 2 * d->hb + 1;
  d->amax = 2 * D.s + 1;
  d->pmax = 2 * D.s + 1 + D.p + 1;
  d->nloc = 2 * D.s + 2;
  d->nq = D.n_quad;
  d->h = (D.hi - D.lo) / (D.n - 1);
  d->stream = (cudaStream_t)stream;
  gauss_legendre01(d->nq, d->gq_t, d->gq_w);
  int st = assemble_impl(d);
  if (st != TAPS_OK) {
    taps_dim_destroy(d);
    return st;
  }
  *out = d;
  return TAPS_OK;
}

extern "C" int taps_dim_info(const taps_dim* d, int* n_all, int* n_free, int* half_band) {
  if (!d) return TAPS_ERR_INVALID_ARG;
  if (n_all) *n_all = d->n;
  if (n_free) *n_free = d->nf;
  if (half_band) *half_band = d->hb;
  return TAPS_OK;
}

extern "C" int taps_dim_copy_band(const taps_dim* d, int op, double* host_out) {
  if (!d || !host_out || op < 0 || op >= TAPS_NUM_OPS) return TAPS_ERR_INVALID_ARG;
  size_t cnt = (size_t)d->nf * d->nb;
  TAPS_CUDA(cudaMemcpyAsync(host_out, d->d_band + op * cnt, cnt * sizeof(double),
                            cudaMemcpyDeviceToHost, d->stream));
  TAPS_CUDA(cudaStreamSynchronize(d->stream));
  return TAPS_OK;
}

extern "C" int taps_dim_copy_shape(const taps_dim* d, double* N_out, double* B_out, double* x_out) {
  if (!d) return TAPS_ERR_INVALID_ARG;
  size_t cnt = (size_t)(d->n - 1) * d->nq * d->nloc;
  if (N_out)
    TAPS_CUDA(cudaMemcpyAsync(N_out, d->d_N, cnt * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  if (B_out)
    TAPS_CUDA(cudaMemcpyAsync(B_out, d->d_B, cnt * sizeof(double), cudaMemcpyDeviceToHost, d->stream));
  if (x_out)
    TAPS_CUDA(cudaMemcpyAsync(x_out, d->d_xq, (size_t)(d->n - 1) * d->nq * sizeof(double),
                              cudaMemcpyDeviceToHost, d->stream));
  TAPS_CUDA(cudaStreamSynchronize(d->stream));
  return TAPS_OK;
}

// Source projection of one factor onto the free nodes of an assembled dimension.
int taps_project_source(const taps_dim* d, int kind, const double* par, const double* nodal_host,
                        double* d_q_free, cudaStream_t s) {
  if (kind < TAPS_SRC_CONST || kind > TAPS_SRC_OPVEC_FULL) return TAPS_ERR_INVALID_ARG;
  DimParams P = make_params(d);
  double* d_nodal = nullptr;
  if (kind == TAPS_SRC_NODAL || kind == TAPS_SRC_OPVEC || kind == TAPS_SRC_OPVEC_FULL) {
    if (!nodal_host) return TAPS_ERR_INVALID_ARG;
    size_t len = kind == TAPS_SRC_OPVEC ? d->nf : d->n;
    TAPS_TRY(taps_alloc((void**)&d_nodal, sizeof(double) * len));
    TAPS_CUDA(cudaMemcpyAsync(d_nodal, nodal_host, sizeof(double) * len, cudaMemcpyHostToDevice, s));
  }
  source_kernel<<<(d->nf + 127) / 128, 128, 0, s>>>(P, d->d_N, d->d_xq, d->d_band_full, d->d_band, kind,
                                                     par[0], par[1], par[2], par[3], d_nodal, d_q_free);
  cudaError_t e = cudaGetLastError();
  if (d_nodal) {
    cudaStreamSynchronize(s);
    cudaFree(d_nodal);
  }
  TAPS_CUDA(e);
  return TAPS_OK;
}

// Projections of every source factor of dim `dimIndex` onto the free nodes, into
// d_q [Rf][nf]: the nodal data of all sources travel in one host-to-device copy
// and one launch projects them all.
int taps_project_sources_dim(const taps_dim* d, const taps_source* sources, int Rf, int dimIndex, double* d_q,
                             cudaStream_t s) {
  DimParams P = make_params(d);
  std::vector<int> kinds(Rf);
  std::vector<long long> offs(Rf, -1);
  size_t tot = 0;
  for (int r = 0; r < Rf; ++r) {
    const int k = sources[r].kind[dimIndex];
    if (k < TAPS_SRC_CONST || k > TAPS_SRC_OPVEC_FULL) return TAPS_ERR_INVALID_ARG;
    kinds[r] = k;
    if (k == TAPS_SRC_NODAL || k == TAPS_SRC_OPVEC || k == TAPS_SRC_OPVEC_FULL) {
      if (!sources[r].nodal[dimIndex]) return TAPS_ERR_INVALID_ARG;
      offs[r] = (long long)tot;
      tot += k == TAPS_SRC_OPVEC ? d->nf : d->n;
    }
  }
  // packed: pars [Rf][4] | nodal data | offsets | kinds
  const size_t npar = 4 * (size_t)Rf;
  const size_t bytes = sizeof(double) * (npar + tot) + sizeof(long long) * Rf + sizeof(int) * Rf;
  std::vector<unsigned char> host(bytes);
  double* hp = reinterpret_cast<double*>(host.data());
  for (int r = 0; r < Rf; ++r)
    for (int j = 0; j < 4; ++j) hp[4 * (size_t)r + j] = sources[r].par[dimIndex][j];
  for (int r = 0; r < Rf; ++r)
    if (offs[r] >= 0) {
      const size_t len = kinds[r] == TAPS_SRC_OPVEC ? d->nf : d->n;
      memcpy(hp + npar + offs[r], sources[r].nodal[dimIndex], sizeof(double) * len);
    }
  memcpy(host.data() + sizeof(double) * (npar + tot), offs.data(), sizeof(long long) * Rf);
  memcpy(host.data() + sizeof(double) * (npar + tot) + sizeof(long long) * Rf, kinds.data(), sizeof(int) * Rf);
  unsigned char* dev = nullptr;
  TAPS_TRY(taps_alloc((void**)&dev, bytes));
  int st = TAPS_OK;
  if (cudaMemcpyAsync(dev, host.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    st = TAPS_ERR_CUDA;
  } else {
    const double* dpars = reinterpret_cast<const double*>(dev);
    const double* dnodal = dpars + npar;
    const long long* doffs = reinterpret_cast<const long long*>(dev + sizeof(double) * (npar + tot));
    const int* dkinds = reinterpret_cast<const int*>(dev + sizeof(double) * (npar + tot) + sizeof(long long) * Rf);
    source_all_kernel<<<dim3((d->nf + 127) / 128, Rf), 128, 0, s>>>(P, d->d_N, d->d_xq, d->d_band_full, d->d_band,
                                                                    dkinds, dpars, doffs, dnodal, d_q);
    if (cudaGetLastError() != cudaSuccess) st = TAPS_ERR_CUDA;
  }
  cudaStreamSynchronize(s);   // the host staging buffer is released on return
  cudaFree(dev);
  return st;
}

// Device-side evaluation of all shape functions of element e at x (point evaluation,
// Eq. 13).  Writes N~ of the nloc local nodes (local k <-> global e - s + k).
__device__ void taps_shape_at(const DimParams& P, const double* ginv, int e, double x, double* N) {
  double xe0 = node_x(P, e), xe1 = node_x(P, e + 1);
  double he = xe1 - xe0;
  for (int k = 0; k < P.nloc; ++k) N[k] = 0.0;
  double hat[2] = {(xe1 - x) / he, (x - xe0) / he};
  double h = P.step;
  for (int c = 0; c < 2; ++c) {
    int i = e + c;
    int j0 = max(0, i - P.s), j1 = min(P.n - 1, i + P.s);
    int na = j1 - j0 + 1, np = na + P.p + 1;
    double row[PMAXC];
    for (int r = 0; r < na; ++r) row[r] = spline_phi(fabs(x - node_x(P, j0 + r)) / (P.a * h));
    double t = (x - node_x(P, i)) / h, pw = 1.0;
    for (int q = 0; q <= P.p; ++q) { row[na + q] = pw; pw *= t; }
    const double* Gi = ginv + (size_t)i * P.amax * P.pmax;
    for (int r = 0; r < na; ++r) {
      double W = 0.0;
      for (int l = 0; l < np; ++l) W += Gi[r * P.pmax + l] * row[l];
      N[(j0 + r) - (e - P.s)] += hat[c] * W;
    }
  }
}

struct PointDims {
  DimParams P[TAPS_MAX_DIMS];
  const double* ginv[TAPS_MAX_DIMS];
  const double* U[TAPS_MAX_DIMS];
};

// One thread per point: u = sum_m prod_d (sum_k N~_k(x_d) U_d[k, m]) with the rows of
// constrained nodes taken as 0.
__global__ void eval_points_kernel(PointDims PD, int D, int M, int n_pts, const double* pts,
                                   double* out) {
  int ip = blockIdx.x * blockDim.x + threadIdx.x;
  if (ip >= n_pts) return;
  double acc[TAPS_MAX_M];
  for (int m = 0; m < M; ++m) acc[m] = 1.0;
  for (int d = 0; d < D; ++d) {
    const DimParams& P = PD.P[d];
    double x = pts[(size_t)ip * D + d];
    x = fmin(fmax(x, P.lo), P.hi);
    int e = (int)floor((x - P.lo) / P.step);
    e = min(max(e, 0), P.n - 2);
    double N[2 * TAPS_MAX_S + 2];
    taps_shape_at(P, PD.ginv[d], e, x, N);
    for (int m = 0; m < M; ++m) {
      double v = 0.0;
      for (int k = 0; k < P.nloc; ++k) {
        int j = e - P.s + k;
        int fj = j - P.off;
        if (j >= 0 && j < P.n && fj >= 0 && fj < P.nf) v += N[k] * PD.U[d][(size_t)m * P.nf + fj];
      }
      acc[m] *= v;
    }
  }
  double u = 0.0;
  for (int m = 0; m < M; ++m) u += acc[m];
  out[ip] = u;
}

extern "C" int taps_eval_points(const taps_problem* prob, const taps_factors* U, int n_pts,
                                const double* pts_dev, double* out_dev) {
  if (!prob || !U || n_pts < 0 || (n_pts > 0 && (!pts_dev || !out_dev))) return TAPS_ERR_INVALID_ARG;
  if (n_pts == 0) return TAPS_OK;
  PointDims PD;
  memset(&PD, 0, sizeof(PD));
  for (int d = 0; d < prob->D; ++d) {
    PD.P[d] = make_params(prob->dims[d]);
    PD.ginv[d] = prob->dims[d]->d_ginv;
    PD.U[d] = U->d_U[d];
  }
  eval_points_kernel<<<(n_pts + 127) / 128, 128, 0, prob->stream>>>(PD, prob->D, U->M, n_pts,
                                                                     pts_dev, out_dev);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

// Weighted operators of dim d: for each j < count with slot[j] >= 0, base[j] (K, M or
// G) weighted by row j of d_w (device, [count][n] all-node values) into band slot
// slot[j] of bands ([slots][nf][nb], device), in one launch on `stream`.
int taps_dim_weighted_bands(const taps_dim* d, int count, const int* base, const int* slot, const double* d_w,
                            double* bands, cudaStream_t stream) {
  if (!d || !d_w || !bands || count < 0) return TAPS_ERR_INVALID_ARG;
  WeightedOps ops;
  memset(&ops, 0, sizeof(ops));
  for (int j = 0; j < count; ++j) {
    if (slot[j] < 0) continue;
    if (ops.count >= TAPS_MAX_SLOTS) return TAPS_ERR_INVALID_ARG;
    if (base[j] != TAPS_OP_K && base[j] != TAPS_OP_M && base[j] != TAPS_OP_G) return TAPS_ERR_INVALID_ARG;
    ops.base[ops.count] = base[j];
    ops.wrow[ops.count] = j;
    ops.slot[ops.count] = slot[j];
    ++ops.count;
  }
  const long long tot = (long long)d->nf * d->nb;
  if (tot == 0 || ops.count == 0) return TAPS_OK;
  DimParams P = make_params(d);
  weighted_band_kernel<<<dim3((unsigned)((tot + 127) / 128), ops.count), 128, 0, stream>>>(P, d->d_N, d->d_B, ops,
                                                                                        d_w, bands);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}
