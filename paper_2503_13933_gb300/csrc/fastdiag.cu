// Fast-diagonalisation reduced solver (Sec. 2.6: the subspace system of one dimension
// is a generalised Sylvester equation, solved by fast diagonalisation).
//
// For a dimension whose distinct operators form a symmetric-definite pencil (A, B)
// (e.g. stiffness K and mass M; or a single SPD operator B, A = 0), the pencil is
// diagonalised once: Phi^T B Phi = I, Phi^T A Phi = diag(mu).  The reduced system
//     A U C_A^T + B U C_B^T = F        (U: n x M, C: M x M, possibly nonsymmetric)
// becomes, with U = Phi Y and G = Phi^T F, n independent M x M systems
//     (mu_i C_A + C_B) Y[i,:]^T = G[i,:]^T,
// so a solve costs two n x n x M products and n small LU solves instead of a
// sequential block elimination over the n block rows.
//
// The one-off pencil decomposition, in FP64: banded Cholesky B = L L^T and
// S = L^{-1} A L^{-T} in one CTA, Householder tridiagonalisation S = Q T Q^T on one
// thread-block cluster; then, in parallel, the eigenvalues of T by Sturm-count multisection (one warp per
// eigenvalue), its eigenvectors by inverse iteration (one thread per eigenvector, one
// per cluster of nearly equal eigenvalues), one step of symmetric orthogonalisation,
// the back-transform Z = Q Z_T (one warp per column), and Phi = L^{-T} Z (one thread per
// column).
#include <string.h>

#include <algorithm>

#include <cooperative_groups.h>

#include "taps_internal.cuh"

#define FD_THREADS 1024

__global__ void fd_dense_kernel(const double* __restrict__ bandA, const double* __restrict__ bandB, int n,
                                int hb, double* __restrict__ A, double* __restrict__ B) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  int i = idx / n, j = idx % n, k = j - i + hb, nb = 2 * hb + 1;
  bool in = (k >= 0 && k < nb);
  A[idx] = (bandA && in) ? bandA[(size_t)i * nb + k] : 0.0;
  B[idx] = in ? bandB[(size_t)i * nb + k] : 0.0;
}

// Single-CTA part of the pencil decomposition: on exit B holds the banded Cholesky
// factor L (lower).  S = L^{-1} A L^{-T} follows in fd_lsolve_kernel (twice) and
// fd_symmetrize_kernel, column-parallel over many CTAs.
__global__ void __launch_bounds__(FD_THREADS) fd_setup_kernel(double* B, int n, int hb, int* status) {
  const int tid = threadIdx.x, nt = blockDim.x;
#define AT(M_, i, j) M_[(size_t)(i) * n + (j)]

  // ---- 1. banded Cholesky of B (lower factor in place; band half-width hb)
  for (int k = 0; k < n; ++k) {
    if (tid == 0) {
      double piv = AT(B, k, k);
      if (!(piv > 0.0) || !isfinite(piv)) {
        taps_flag(status, TAPS_DEV_SINGULAR);
        piv = 1.0;
      }
      AT(B, k, k) = sqrt(piv);
    }
    __syncthreads();
    double lkk = AT(B, k, k);
    int top = min(n - 1, k + hb);
    for (int i = k + 1 + tid; i <= top; i += nt) AT(B, i, k) /= lkk;
    __syncthreads();
    int w = top - k;
    for (int idx = tid; idx < w * w; idx += nt) {
      int i = k + 1 + idx / w, j = k + 1 + idx % w;
      if (j <= i) AT(B, i, j) -= AT(B, i, k) * AT(B, j, k);
    }
    __syncthreads();
  }

#undef AT
}

// Out[:, c] = L^{-1} (In[:, c] or, with transposed input, In[c, :]^T) for the banded
// lower factor L (half-bandwidth hb): one thread per column c, the chain of n
// substitutions with the diagonal's reciprocal; 32-thread CTAs spread the columns over
// the SMs (each chain is FP64-latency bound).
__global__ void __launch_bounds__(32) fd_lsolve_kernel(const double* __restrict__ L, const double* __restrict__ In,
                                                       int n, int hb, int trans_in, double* __restrict__ Out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = 0; i < n; ++i) {
    double s = trans_in ? In[(size_t)c * n + i] : In[(size_t)i * n + c];
    for (int j = max(0, i - hb); j < i; ++j) s -= L[(size_t)i * n + j] * Out[(size_t)j * n + c];
    Out[(size_t)i * n + c] = s * taps_rcp(L[(size_t)i * n + i]);
  }
}

// A = (V + V^T) / 2
__global__ void fd_symmetrize_kernel(const double* __restrict__ V, int n, double* __restrict__ A) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx % n);
  A[idx] = 0.5 * (V[(size_t)i * n + j] + V[(size_t)j * n + i]);
}

// ---------------------------------------------------------------------------------
// Householder tridiagonalisation S = Q T Q^T of the symmetric S held in A (n x n,
// row-major), on one cluster of NC CTAs (16 where the GPU can place a 16-CTA cluster,
// else 8; the arithmetic is the same for both) with hardware cluster barriers between
// the phases of a step.  Step k: every CTA stages column k below the diagonal in
// shared memory and forms the same reflector v (beta = 2 / v.v); one warp per row of
// the cluster computes p = beta S22 v; after a cluster barrier every CTA forms
// w = p - (beta v.p / 2) v and its warps update their rows of S22 -= v w^T + w v^T;
// a second barrier ends the step.  Values written by other CTAs are read through L2.
// On exit (d, e) hold T (e[i] couples i and i+1), the rows of V the reflectors
// (row k: entries k+1 .. n-1) and beta their factors.
// ---------------------------------------------------------------------------------
#define TD_THREADS 1024
__device__ __forceinline__ void td_cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

template <int NC>
__global__ void __launch_bounds__(TD_THREADS)
    fd_tridiag_kernel(double* __restrict__ A, double* __restrict__ V, double* __restrict__ p,
                      double* __restrict__ beta, double* __restrict__ d, double* __restrict__ e, int n) {
  extern __shared__ double tds[];   // v [n], p [n], w [n]
  __shared__ double red[32];
  double* vs = tds;
  double* ps = tds + n;
  double* ws = tds + 2 * n;
  const int rank = blockIdx.x;   // the grid is one cluster
  const int tid = threadIdx.x, lane = tid & 31;
  const int gwarp = rank * (TD_THREADS / 32) + (tid >> 5);
  const int nwarps = NC * (TD_THREADS / 32);
#define AT(i, j) A[(size_t)(i) * n + (j)]
  for (int k = 0; k + 2 < n; ++k) {
    const int len = n - k - 1;
    double s2 = 0.0;
    for (int t = tid; t < len; t += TD_THREADS) {
      const double x = __ldcg(&AT(k + 1 + t, k));
      vs[t] = x;
      s2 += x * x;
    }
    s2 = block_sum(s2, red);   // also orders the vs writes
    if (s2 == 0.0) {           // the same in every CTA: nothing to reflect
      if (rank == 0 && tid == 0) {
        beta[k] = 0.0;
        d[k] = __ldcg(&AT(k, k));
        e[k] = 0.0;
      }
      continue;
    }
    const double x0 = vs[0];
    const double alpha = -copysign(sqrt(s2), x0);
    const double v0 = x0 - alpha;
    const double bk = 2.0 / (s2 - x0 * x0 + v0 * v0);
    __syncthreads();
    if (tid == 0) vs[0] = v0;
    __syncthreads();
    // p = beta S22 v, one warp per row
    for (int i = gwarp; i < len; i += nwarps) {
      const double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      double acc = 0.0;
      for (int t = lane; t < len; t += 32) acc += __ldcg(row + t) * vs[t];
      acc = warp_sum(acc);
      if (lane == 0) p[i] = bk * acc;
    }
    td_cluster_sync();
    double pv = 0.0;
    for (int t = tid; t < len; t += TD_THREADS) {
      const double pt = __ldcg(p + t);
      ps[t] = pt;
      pv += pt * vs[t];
    }
    pv = block_sum(pv, red);
    const double Kc = 0.5 * bk * pv;
    for (int t = tid; t < len; t += TD_THREADS) ws[t] = ps[t] - Kc * vs[t];
    __syncthreads();
    for (int i = gwarp; i < len; i += nwarps) {
      double* row = A + (size_t)(k + 1 + i) * n + (k + 1);
      const double vi = vs[i], wi = ws[i];
      for (int t = lane; t < len; t += 32) row[t] = __ldcg(row + t) - (vi * ws[t] + wi * vs[t]);
    }
    if (rank == 0) {
      for (int t = tid; t < len; t += TD_THREADS) V[(size_t)k * n + k + 1 + t] = vs[t];
      if (tid == 0) {
        beta[k] = bk;
        d[k] = __ldcg(&AT(k, k));
        e[k] = alpha;
      }
    }
    td_cluster_sync();
  }
  if (rank == 0 && tid == 0) {
    if (n >= 2) {
      d[n - 2] = __ldcg(&AT(n - 2, n - 2));
      e[n - 2] = __ldcg(&AT(n - 1, n - 2));
    }
    d[n - 1] = __ldcg(&AT(n - 1, n - 1));
    e[n - 1] = 0.0;
    for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) beta[k] = 0.0;
  }
#undef AT
}

// The same tridiagonalisation with S held in the cluster's distributed shared memory
// (n small enough that ceil(n / NC) rows of n doubles fit one CTA's shared memory):
// CTA r keeps rows i = r, r + NC, ...  Step k: every CTA gathers column k from the
// rows' owners (remote shared-memory loads), forms the reflector, computes p_i for its
// own rows and stores each p_i into every CTA's copy of p; after a cluster barrier
// every CTA forms w and updates its own rows; a second barrier ends the step.  S never
// leaves shared memory.
template <int NC>
__global__ void __launch_bounds__(TD_THREADS)
    fd_tridiag_dsmem_kernel(const double* __restrict__ A, double* __restrict__ V, double* __restrict__ beta,
                            double* __restrict__ d, double* __restrict__ e, int n) {
  extern __shared__ double tsm[];   // vs [n] | ps [n] | ws [n] | own rows [nr][n]
  __shared__ double red[32];
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nwarps = TD_THREADS / 32;
  double* vs = tsm;
  double* ps = tsm + n;
  double* ws = tsm + 2 * n;
  double* rows = tsm + 3 * n;
  const int nr = (n - rank + NC - 1) / NC;   // rows i = rank + NC * l, l < nr
  for (long long idx = tid; idx < (long long)nr * n; idx += TD_THREADS) {
    const int l = (int)(idx / n), j = (int)(idx % n);
    rows[(size_t)l * n + j] = A[(size_t)(rank + NC * l) * n + j];
  }
  cluster.sync();
  for (int k = 0; k + 2 < n; ++k) {
    const int len = n - k - 1;
    // column k below the diagonal, from the owners of its rows
    double s2 = 0.0;
    for (int t = tid; t < len; t += TD_THREADS) {
      const int i = k + 1 + t;
      const double* owner_rows = cluster.map_shared_rank(rows, i % NC);
      const double x = owner_rows[(size_t)(i / NC) * n + k];
      vs[t] = x;
      s2 += x * x;
    }
    s2 = block_sum(s2, red);
    if (s2 == 0.0) {   // the same in every CTA
      if (k % NC == rank && tid == 0) d[k] = rows[(size_t)(k / NC) * n + k];
      if (rank == 0 && tid == 0) {
        beta[k] = 0.0;
        e[k] = 0.0;
      }
      cluster.sync();
      continue;
    }
    const double x0 = vs[0];
    const double alpha = -copysign(sqrt(s2), x0);
    const double v0 = x0 - alpha;
    const double bk = 2.0 / (s2 - x0 * x0 + v0 * v0);
    __syncthreads();
    if (tid == 0) vs[0] = v0;
    __syncthreads();
    // p_i for own rows i >= k + 1, pushed into every CTA's ps
    const int l0 = (k + 1 - rank + NC - 1) / NC;   // first own row >= k + 1
    for (int l = l0 + warp; l < nr; l += nwarps) {
      const int i = rank + NC * l;
      const double* row = rows + (size_t)l * n + (k + 1);
      double acc = 0.0;
      for (int t = lane; t < len; t += 32) acc += row[t] * vs[t];
      acc = warp_sum(acc) * bk;
      if (lane < NC) cluster.map_shared_rank(ps, lane)[i - k - 1] = acc;
    }
    cluster.sync();
    double pv = 0.0;
    for (int t = tid; t < len; t += TD_THREADS) pv += ps[t] * vs[t];
    pv = block_sum(pv, red);
    const double Kc = 0.5 * bk * pv;
    for (int t = tid; t < len; t += TD_THREADS) ws[t] = ps[t] - Kc * vs[t];
    __syncthreads();
    for (int l = l0 + warp; l < nr; l += nwarps) {
      const int i = rank + NC * l - (k + 1);   // index within the trailing block
      double* row = rows + (size_t)l * n + (k + 1);
      const double vi = vs[i], wi = ws[i];
      for (int t = lane; t < len; t += 32) row[t] -= vi * ws[t] + wi * vs[t];
    }
    if (rank == 0) {
      for (int t = tid; t < len; t += TD_THREADS) V[(size_t)k * n + k + 1 + t] = vs[t];
      if (tid == 0) {
        beta[k] = bk;
        e[k] = alpha;
      }
    }
    if (k % NC == rank && tid == 0) d[k] = rows[(size_t)(k / NC) * n + k];
    cluster.sync();
  }
  if (tid == 0) {
    for (int i = (n >= 2 ? n - 2 : 0); i < n; ++i)
      if (i % NC == rank) d[i] = rows[(size_t)(i / NC) * n + i];
    if (n >= 2 && (n - 1) % NC == rank) e[n - 2] = rows[(size_t)((n - 1) / NC) * n + (n - 2)];
    if (rank == 0) {
      e[n - 1] = 0.0;
      for (int k = (n >= 2 ? n - 2 : 0); k < n; ++k) beta[k] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------------
// Eigenvalues of the symmetric tridiagonal T (diagonal d, off-diagonal e) by Sturm-count
// multisection: warp k finds the k-th smallest eigenvalue.  Each lane counts the
// eigenvalues below one of 32 interior points of the current interval (Sturm count);
// the first point whose count exceeds k bounds the eigenvalue from above, its left
// neighbour from below, so each round shrinks the interval 33x.  The start interval is
// Gershgorin's; it is refined to a width of 4 eps ||T|| (what Sturm counts resolve),
// about 11 rounds, or until rounding stops it shrinking.
// ---------------------------------------------------------------------------------
// Number of eigenvalues of T below x: the negative pivots of T - x I,
// q_i = (d_i - x) - e_{i-1}^2 / q_{i-1}; a pivot smaller than pivmin counts as -pivmin.
__device__ __forceinline__ int fd_sturm_count(const double* __restrict__ d, const double* __restrict__ e,
                                              int n, double x, double pivmin) {
  double q = d[0] - x;
  if (fabs(q) < pivmin) q = -pivmin;
  int cnt = q < 0.0 ? 1 : 0;
#pragma unroll 4
  for (int i = 1; i < n; ++i) {
    const double ei = e[i - 1];
    q = (d[i] - x) - (ei * ei) * taps_rcp(q);
    if (fabs(q) < pivmin) q = -pivmin;
    cnt += q < 0.0 ? 1 : 0;
  }
  return cnt;
}

__global__ void fd_bisect_kernel(const double* __restrict__ d, const double* __restrict__ e, int n,
                                 double* __restrict__ lam) {
  const int k = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= n) return;   // whole warps
  double lo = INFINITY, hi = -INFINITY, e2max = 0.0;
  for (int i = lane; i < n; i += 32) {
    const double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i < n - 1 ? fabs(e[i]) : 0.0);
    lo = fmin(lo, d[i] - r);
    hi = fmax(hi, d[i] + r);
    if (i < n - 1) e2max = fmax(e2max, e[i] * e[i]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
    hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    e2max = fmax(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
  }
  const double eps = 2.220446049250313e-16;
  const double tnorm = fmax(fabs(lo), fabs(hi));
  // underflow guard for the Sturm pivots (the smallest normal double times the largest
  // squared off-diagonal), small enough not to limit the eigenvalues' accuracy
  const double pivmin = 2.2250738585072014e-308 * fmax(1.0, e2max);
  lo -= 4.0 * eps * tnorm + pivmin;
  hi += 4.0 * eps * tnorm + pivmin;
  double wprev = INFINITY;
  for (int it = 0; it < 40; ++it) {
    const double w = hi - lo;
    // Sturm counts resolve an eigenvalue to about eps ||T|| (absolute)
    if (w <= 4.0 * eps * tnorm + pivmin) break;
    if (it > 0 && !(w < wprev)) break;   // rounding no longer separates the trial points
    wprev = w;
    const double x = lo + w * (double)(lane + 1) / 33.0;
    const unsigned above = __ballot_sync(0xffffffffu, fd_sturm_count(d, e, n, x, pivmin) > k);
    const int j = above ? __ffs(above) - 1 : 32;
    const double nhi = (j < 32) ? lo + w * (double)(j + 1) / 33.0 : hi;
    const double nlo = (j > 0) ? lo + w * (double)j / 33.0 : lo;
    lo = nlo;
    hi = nhi;
  }
  if (lane == 0) lam[k] = 0.5 * (lo + hi);
}

// ---------------------------------------------------------------------------------
// Eigenvectors of T by inverse iteration: thread k factors T - lam_k I by Gaussian
// elimination with partial pivoting (U has two super-diagonals) and solves three times
// from a fixed start vector, normalising after each solve.  Eigenvalues closer than
// 1e-5 ||T|| form a cluster, handled in order by the thread of its first member, each
// iterate orthogonalised against the members already done (modified Gram-Schmidt).
// Z is n x n row-major (column k = eigenvector k); W holds five n x n arrays laid out
// [array][row][k] so that neighbouring threads touch neighbouring words.
// ---------------------------------------------------------------------------------
__global__ void fd_invit_kernel(const double* __restrict__ d, const double* __restrict__ e,
                                const double* __restrict__ lam, int n, double* __restrict__ Z,
                                double* __restrict__ W) {
  const int k0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (k0 >= n) return;
  double tnorm = 0.0;   // Gershgorin bound of ||T||
  for (int i = 0; i < n; ++i)
    tnorm = fmax(tnorm, fabs(d[i]) + (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0));
  if (!(tnorm > 0.0)) tnorm = 1.0;
  const double ctol = 1e-5 * tnorm;
  if (k0 > 0 && lam[k0] - lam[k0 - 1] <= ctol) return;   // not the first member of its cluster
  int k1 = k0;
  while (k1 + 1 < n && lam[k1 + 1] - lam[k1] <= ctol) ++k1;
  const double tiny = 2.220446049250313e-16 * tnorm;
  const size_t nn = (size_t)n * n;
#define WA(a, i) W[(size_t)(a) * nn + (size_t)(i) * n + k]
#define ZC(i) Z[(size_t)(i) * n + k]
  for (int k = k0; k <= k1; ++k) {
    const double lk = lam[k];
    // ---- factor T - lk I: arrays 0: 1/U0, 1: U1, 2: U2, 3: multiplier, 4: row swap
    double ai = d[0] - lk, bi = n > 1 ? e[0] : 0.0;
    for (int i = 0; i + 1 < n; ++i) {
      const double ci = e[i], an = d[i + 1] - lk, bn = (i + 2 < n) ? e[i + 1] : 0.0;
      if (fabs(ai) >= fabs(ci)) {
        if (ai == 0.0) ai = tiny;
        const double m = ci / ai;
        WA(0, i) = 1.0 / ai;
        WA(1, i) = bi;
        WA(2, i) = 0.0;
        WA(3, i) = m;
        WA(4, i) = 0.0;
        ai = an - m * bi;
        bi = bn;
      } else {
        const double m = ai / ci;
        WA(0, i) = 1.0 / ci;
        WA(1, i) = an;
        WA(2, i) = bn;
        WA(3, i) = m;
        WA(4, i) = 1.0;
        ai = bi - m * an;
        bi = -m * bn;
      }
    }
    if (ai == 0.0) ai = tiny;
    WA(0, n - 1) = 1.0 / ai;
    WA(1, n - 1) = 0.0;   // the last row has no super-diagonals
    WA(2, n - 1) = 0.0;
    // ---- start vector (fixed, different per k), then three solves
    for (int i = 0; i < n; ++i) ZC(i) = 1.0 + 0.5 * sin(0.7 * i + 1.3 * k);
    for (int it = 0; it < 3; ++it) {
      // forward: row swaps and multipliers (the running entry stays in a register)
      double yi = ZC(0);
#pragma unroll 8
      for (int i = 0; i + 1 < n; ++i) {
        double yn = ZC(i + 1);
        if (WA(4, i) != 0.0) {
          const double t = yi;
          yi = yn;
          yn = t;
        }
        ZC(i) = yi;
        yi = yn - WA(3, i) * yi;
      }
      ZC(n - 1) = yi;
      // backward with the two super-diagonals (z_{i+1}, z_{i+2} in registers)
      double z1 = 0.0, z2 = 0.0;
#pragma unroll 8
      for (int i = n - 1; i >= 0; --i) {
        const double zi = (ZC(i) - WA(1, i) * z1 - WA(2, i) * z2) * WA(0, i);
        ZC(i) = zi;
        z2 = z1;
        z1 = zi;
      }
      for (int j = k0; j < k; ++j) {   // against the cluster's earlier members
        double dot = 0.0;
        for (int i = 0; i < n; ++i) dot += Z[(size_t)i * n + j] * ZC(i);
        for (int i = 0; i < n; ++i) ZC(i) -= dot * Z[(size_t)i * n + j];
      }
      double nrm = 0.0;
      for (int i = 0; i < n; ++i) nrm += ZC(i) * ZC(i);
      const double inv = (nrm > 0.0) ? 1.0 / sqrt(nrm) : 0.0;
      for (int i = 0; i < n; ++i) ZC(i) *= inv;
    }
  }
#undef WA
#undef ZC
}

// ---------------------------------------------------------------------------------
// Symmetric orthogonalisation of the inverse-iteration vectors, first order:
// Z <- Z - Z E / 2 with E = Z^T Z - I.  Independently computed eigenvectors are
// orthogonal only to ~eps ||T|| / gap (1e-11 for the lowest eigenvalues of a stiffness
// pencil); one step squares that, and Z^T T Z stays diagonal to ~eps ||T|| because the
// correction of entry (j, k) is scaled by lam_j + lam_k.  E[j][k]: one thread each;
// four partial sums shorten the dependent FP64 chain.
// ---------------------------------------------------------------------------------
__global__ void fd_gram_minus_identity_kernel(const double* __restrict__ Z, int n, double* __restrict__ E) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int j = (int)(idx / n), k = (int)(idx % n);
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int i = 0;
  for (; i + 3 < n; i += 4) {
    a0 += Z[(size_t)i * n + j] * Z[(size_t)i * n + k];
    a1 += Z[(size_t)(i + 1) * n + j] * Z[(size_t)(i + 1) * n + k];
    a2 += Z[(size_t)(i + 2) * n + j] * Z[(size_t)(i + 2) * n + k];
    a3 += Z[(size_t)(i + 3) * n + j] * Z[(size_t)(i + 3) * n + k];
  }
  for (; i < n; ++i) a0 += Z[(size_t)i * n + j] * Z[(size_t)i * n + k];
  E[idx] = ((a0 + a1) + (a2 + a3)) - (j == k ? 1.0 : 0.0);
}

__global__ void fd_orth_update_kernel(const double* __restrict__ Z, const double* __restrict__ E, int n,
                                      double* __restrict__ Zout) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), k = (int)(idx % n);
  const double* zi = Z + (size_t)i * n;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  int j = 0;
  for (; j + 3 < n; j += 4) {
    a0 += zi[j] * E[(size_t)j * n + k];
    a1 += zi[j + 1] * E[(size_t)(j + 1) * n + k];
    a2 += zi[j + 2] * E[(size_t)(j + 2) * n + k];
    a3 += zi[j + 3] * E[(size_t)(j + 3) * n + k];
  }
  for (; j < n; ++j) a0 += zi[j] * E[(size_t)j * n + k];
  Zout[idx] = zi[k] - 0.5 * ((a0 + a1) + (a2 + a3));
}

// ---------------------------------------------------------------------------------
// Back-transform Z <- Q Z with Q = H_0 H_1 ... H_{n-3}, H_r = I - beta_r v_r v_r^T acting
// on rows r+1 .. n-1 (v_r in row r of V): warp c takes column c through the reflections
// from the last to the first, the column held in shared memory.
// ---------------------------------------------------------------------------------
__global__ void fd_backtransform_kernel(const double* __restrict__ V, const double* __restrict__ beta, int n,
                                        double* __restrict__ Z) {
  extern __shared__ double zs[];   // [warps per CTA][n]
  const int wl = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int c = blockIdx.x * (blockDim.x >> 5) + wl;
  if (c >= n) return;   // whole warps
  double* z = zs + (size_t)wl * n;
  for (int i = lane; i < n; i += 32) z[i] = Z[(size_t)i * n + c];
  __syncwarp();
  for (int r = n - 3; r >= 0; --r) {
    const double br = beta[r];
    if (br == 0.0) continue;
    const double* v = V + (size_t)r * n;
    double dot = 0.0;
    for (int i = r + 1 + lane; i < n; i += 32) dot += v[i] * z[i];
    dot = warp_sum(dot) * br;
    for (int i = r + 1 + lane; i < n; i += 32) z[i] -= dot * v[i];
    __syncwarp();
  }
  for (int i = lane; i < n; i += 32) Z[(size_t)i * n + c] = z[i];
}

// Phi = L^{-T} Z (L: the banded Cholesky factor in B, lower, half-width hb), Phi^T, and
// mu = the eigenvalues; one thread per column.  Without an A (single-operator pencil)
// Z = I and mu = 0.
__global__ void fd_phi_kernel(const double* __restrict__ L, const double* __restrict__ Z,
                              const double* __restrict__ lam, int n, int hb, double* __restrict__ Phi,
                              double* __restrict__ PhiT, double* __restrict__ mu, int* status) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  for (int i = n - 1; i >= 0; --i) {
    double sacc = Z ? Z[(size_t)i * n + c] : (i == c ? 1.0 : 0.0);
    for (int j = i + 1; j <= min(n - 1, i + hb); ++j) sacc -= L[(size_t)j * n + i] * Phi[(size_t)j * n + c];
    const double v = sacc * taps_rcp(L[(size_t)i * n + i]);
    Phi[(size_t)i * n + c] = v;
    PhiT[(size_t)c * n + i] = v;
  }
  const double m = lam ? lam[c] : 0.0;
  mu[c] = m;
  if (!isfinite(m)) taps_flag(status, TAPS_DEV_NONFINITE);
}

// ---------------------------------------------------------------------------------
// Per-solve kernels
// ---------------------------------------------------------------------------------
// F[i][m] = sum_r q_r[i] c_r[m]
__global__ void fd_rhs_kernel(const double* __restrict__ q, const double* __restrict__ c, int Rf, int nf,
                              int M, double* __restrict__ F) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nf * M) return;
  int i = idx / M, m = idx % M;
  double v = 0.0;
  for (int r = 0; r < Rf; ++r) v += q[(size_t)r * nf + i] * c[(size_t)r * M + m];
  F[idx] = v;
}

// PQ[r][i] = sum_j PhiT[i][j] q[r][j]: the source vectors of dim d in the eigenbasis
// of its pencil.  The reduced right-hand side of dim d is F = Q c (c from the other
// dims), so its transform Phi^T F = (Phi^T Q) c needs only this fixed n x Rf matrix.
__global__ void fd_pq_kernel(const double* __restrict__ PhiT, const double* __restrict__ q, int n,
                             int Rf, double* __restrict__ PQ) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * Rf) return;
  const int r = (int)(idx / n), i = (int)(idx % n);
  const double* row = PhiT + (size_t)i * n;
  const double* qr = q + (size_t)r * n;
  double acc = 0.0;
  for (int j = 0; j < n; ++j) acc += row[j] * qr[j];
  PQ[idx] = acc;
}

// Out[i][m] = sum_j Mat[i][j] In[j][m] (Mat n x n row-major, In n x M row-major).
// One CTA per output row i.  Its RG_WARPS warps (one per SM sub-partition) split the
// sum over j; within a warp the lanes split it again, each lane keeping 32 mode
// accumulators.  A butterfly reduce-scatter then leaves lane l of each warp with the
// warp's sum for mode l (31 additions per lane instead of a chain of 32), and the
// warps' sums are combined through shared memory.  FP64 on this GPU is issue-bound
// per sub-partition, so spreading one row over all four pipes matters.
// Out is n x M row-major, or (colmajor) the factor layout Out[m * n + i]; in the
// factor layout a non-null Save receives the row's previous values first.
#define RG_WARPS 4
__global__ void __launch_bounds__(RG_WARPS * 32) fd_rowgemm_kernel(const double* __restrict__ Mat,
                                                                   const double* __restrict__ In, int n,
                                                                   int M, double* __restrict__ Out,
                                                                   int colmajor,
                                                                   double* __restrict__ Save) {
  __shared__ double part[RG_WARPS][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int i = blockIdx.x;
  taps_pdl_wait();
  if (colmajor && Save)   // the writes below come after a barrier
    for (int m = threadIdx.x; m < M; m += blockDim.x) Save[(size_t)m * n + i] = Out[(size_t)m * n + i];
  const double* row = Mat + (size_t)i * n;
  const int step = RG_WARPS * 32;
  for (int m0 = 0; m0 < M; m0 += 32) {
    const int mc = min(32, M - m0);
    double acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.0;
    for (int j = warp * 32 + lane; j < n; j += step) {
      const double a = row[j];
      const double* in = In + (size_t)j * M + m0;
#pragma unroll
      for (int c = 0; c < 32; ++c)
        if (c < mc) acc[c] += a * in[c];
    }
    // reduce-scatter: at offset o a lane keeps the half of its current modes selected
    // by lane bit o and receives its partner's values of that half
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      const bool up = (lane & o) != 0;
#pragma unroll
      for (int c = 0; c < o; ++c) {
        const double send = up ? acc[c] : acc[c + o];
        const double keep = up ? acc[c + o] : acc[c];
        acc[c] = keep + __shfl_xor_sync(0xffffffffu, send, o);
      }
    }
    part[warp][lane] = acc[0];   // the warp's sum for mode m0 + lane
    __syncthreads();
    if (threadIdx.x < mc) {
      const double sum = (part[0][threadIdx.x] + part[1][threadIdx.x]) +
                         (part[2][threadIdx.x] + part[3][threadIdx.x]);
      if (colmajor) Out[(size_t)(m0 + threadIdx.x) * n + i] = sum;
      else Out[(size_t)i * M + m0 + threadIdx.x] = sum;
    }
    __syncthreads();
  }
}

// One warp per node i, M <= 32: lane r holds row r of (mu_i C_A + C_B | g_i) in
// registers.  Without refinement: LU without pivoting in FP64 (the systems have a
// positive definite symmetric part) and back substitution by shuffles.  With
// refinement: the LU runs in FP32 (whose dependent-instruction latency is a small
// fraction of FP64's on this GPU) and the solution is refined in FP64
// (y += T^{-1}_32 (g - T y)) until the FP64 residual is at the level of FP64
// rounding; a system that does not get there in 4 steps is solved again by the FP64
// LU.  A zero or non-finite pivot is reported as TAPS_DEV_SINGULAR.
template <typename R>
__device__ __forceinline__ void warp_lu_inplace(R row[33], int lane, int M, bool& bad) {
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    if (p < M) {
      R piv = __shfl_sync(0xffffffffu, row[p], p);
      bad |= !(fabs((double)piv) > 0.0) || !isfinite((double)piv);
      R l = (lane > p && lane < M && piv != (R)0) ? row[p] / piv : (R)0;
#pragma unroll
      for (int c = 0; c < 32; ++c) {
        if (c > p && c < M) {
          R pc = __shfl_sync(0xffffffffu, row[c], p);
          row[c] -= l * pc;
        }
      }
      if (lane > p && lane < M) row[p] = l;   // keep the multiplier (unit lower L)
    }
  }
}

// Solve L U x = b with the factors of warp_lu_inplace; b and x are lane-distributed.
template <typename R>
__device__ __forceinline__ R warp_lu_solve(const R row[33], R b, int lane, int M) {
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    if (p < M) {
      R bp = __shfl_sync(0xffffffffu, b, p);
      if (lane > p && lane < M) b -= row[p] * bp;
    }
  }
  R x = (R)0;
#pragma unroll
  for (int c = 31; c >= 0; --c) {
    if (c < M) {
      R xc = (lane == c && row[c] != (R)0) ? b / row[c] : (R)0;
      xc = __shfl_sync(0xffffffffu, xc, c);
      if (lane == c) x = xc;
      if (lane < c) b -= row[c] * xc;
    }
  }
  return x;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__global__ void __launch_bounds__(32) fd_small_solve_warp_kernel(const double* __restrict__ CA,
                                                                 const double* __restrict__ CB,
                                                                 const double* __restrict__ mu,
                                                                 const double* __restrict__ G, int n,
                                                                 int M, double* __restrict__ Y,
                                                                 int* status, int refine) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x;   // one warp per CTA: the n systems spread over every SM
  if (i >= n) return;
  const double mi = (CA && mu) ? mu[i] : 0.0;
  double row[33];
#pragma unroll
  for (int c = 0; c < 32; ++c) {
    double v = 0.0;
    if (lane < M && c < M) v = (CA ? mi * CA[lane * M + c] : 0.0) + CB[lane * M + c];
    row[c] = v;
  }
  const double g = (lane < M) ? G[(size_t)i * M + lane] : 0.0;
  bool bad = false;
  double x = 0.0;
  bool done = false;
  if (refine) {
    float rf[33];
#pragma unroll
    for (int c = 0; c < 33; ++c) rf[c] = (float)row[c];
    bool bad32 = false;
    warp_lu_inplace<float>(rf, lane, M, bad32);
    if (!bad32) {
      double tnorm = 0.0;
#pragma unroll
      for (int c = 0; c < 32; ++c) tnorm += fabs(row[c]);
      tnorm = warp_max(tnorm);
      double r = g;
      for (int it = 0; it < 4 && !done; ++it) {
        x += (double)warp_lu_solve<float>(rf, (float)r, lane, M);
        // r = g - T x in FP64, as four independent partial sums (FP64 latency is long)
        double a0 = g, a1 = 0.0, a2 = 0.0, a3 = 0.0;
#pragma unroll
        for (int c = 0; c < 32; c += 4) {
          double x0 = __shfl_sync(0xffffffffu, x, c), x1 = __shfl_sync(0xffffffffu, x, c + 1);
          double x2 = __shfl_sync(0xffffffffu, x, c + 2), x3 = __shfl_sync(0xffffffffu, x, c + 3);
          if (c < M) a0 -= row[c] * x0;
          if (c + 1 < M) a1 -= row[c + 1] * x1;
          if (c + 2 < M) a2 -= row[c + 2] * x2;
          if (c + 3 < M) a3 -= row[c + 3] * x3;
        }
        r = (lane < M) ? (a0 + a1) + (a2 + a3) : 0.0;
        double rmax = warp_max(fabs(r)), xmax = warp_max(fabs(x)), gmax = warp_max(fabs(g));
        // FP64 backward accuracy (a few eps), so that the refined path gives the
        // FP64 path's factors; the FP64 LU below is the fallback
        done = rmax <= 8.0 * 2.220446049250313e-16 * (tnorm * xmax + gmax);
        if (!isfinite(rmax)) break;
      }
    }
  }
  if (!done) {   // FP64 LU (also the fallback of the refined path)
    warp_lu_inplace<double>(row, lane, M, bad);
    x = warp_lu_solve<double>(row, g, lane, M);
    if (bad && lane == 0) taps_flag(status, TAPS_DEV_SINGULAR);
  }
  if (lane < M) Y[(size_t)i * M + lane] = x;
}

// One CTA of four warps per node i, M <= 32, FP64.  FP64 instructions issue at a
// fraction of a lane per clock per SM sub-partition on this GPU, so the elimination
// of one system is spread over the four sub-partitions: warp w holds the columns
// c = w, w+4, w+8, ... of T = mu_i C_A + C_B (lane r = row r) and warp 0 also the
// right-hand side g_i = sum_r PQ[r][i] c_r, formed here from the transformed source
// vectors (the warps split the sum over r).  At step p every warp updates its
// columns c > p with the multipliers l_r = T[r][p] / T[p][p] of that step, which the
// owner of column p has published in shared memory (one reciprocal of the pivot,
// kept for the back substitution).  The chain of pivots is the bound: the owner of
// column p+1 updates that column first (its row-p value fetched before the barrier),
// takes the pivot's reciprocal (approximate seed + series refinement) and issues its
// other updates while the reciprocal completes.  No pivoting, as in the one-warp
// solve.  The upper factor then goes to shared memory and warp 0 back-substitutes.
__global__ void __launch_bounds__(128) fd_small_solve_quad_kernel(const double* __restrict__ CA,
                                                                  const double* __restrict__ CB,
                                                                  const double* __restrict__ mu,
                                                                  const double* __restrict__ PQ,
                                                                  const double* __restrict__ cf, int Rf,
                                                                  int n, int M, double* __restrict__ Y,
                                                                  int* status) {
  __shared__ double gpart[4][32];
  __shared__ double lbuf[2][32];
  __shared__ double invd[32];
  __shared__ double Ush[32][33];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int i = blockIdx.x;
  if (i >= n) return;
  taps_pdl_wait();
  const double mi = (CA && mu) ? mu[i] : 0.0;
  double v[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = 4 * k + w;
    double x = 0.0;
    if (lane < M && c < M) x = (CA ? mi * CA[lane * M + c] : 0.0) + CB[lane * M + c];
    v[k] = x;
  }
  double gp = 0.0;
  if (lane < M)
    for (int r = w; r < Rf; r += 4) gp += PQ[(size_t)r * n + i] * cf[(size_t)r * M + lane];
  gpart[w][lane] = gp;
  bool bad = false;
  // multipliers of step 0 (column 0 belongs to warp 0)
  if (w == 0) {
    const double piv = __shfl_sync(0xffffffffu, v[0], 0);
    bad |= !taps_finite_nonzero(piv);
    const double inv = taps_rcp(piv);
    lbuf[0][lane] = (lane > 0 && lane < M) ? v[0] * inv : 0.0;
    if (lane == 0) invd[0] = inv;
  }
  // row 0 of column 1, for the owner of the next pivot
  double pc_next = (w == 1) ? __shfl_sync(0xffffffffu, v[0], 0) : 0.0;
  __syncthreads();
  double b = (w == 0) ? (gpart[0][lane] + gpart[1][lane]) + (gpart[2][lane] + gpart[3][lane]) : 0.0;
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    if (p < M) {
      const double l = lbuf[p & 1][lane];
      const int q = p + 1;   // next pivot column, owned by warp q & 3 in slot q >> 2
      if (q < M && w == (q & 3)) {
        // owner of column q: that column (its row p was fetched before the barrier),
        // the pivot's reciprocal, then its other columns in the same block so that
        // their FP64 issue fills the reciprocal's latency, then the next multipliers
        v[q >> 2] -= l * pc_next;
        const double piv = __shfl_sync(0xffffffffu, v[q >> 2], q);
        const double inv = taps_rcp(piv);
#pragma unroll
        for (int k = (q >> 2) + 1; k < 8; ++k) v[k] -= l * __shfl_sync(0xffffffffu, v[k], p);
        lbuf[q & 1][lane] = (lane > q && lane < M) ? v[q >> 2] * inv : 0.0;
        if (lane == 0) invd[q] = inv;
        bad |= !taps_finite_nonzero(piv);
      } else {
#pragma unroll
        for (int k = 0; k < 8; ++k) {   // this warp's columns c > p
          if (4 * k + 3 <= p) continue;                 // every column of this slot is <= p
          if (4 * k <= p && w <= p - 4 * k) continue;   // column 4k + w <= p
          v[k] -= l * __shfl_sync(0xffffffffu, v[k], p);
        }
      }
      if (w == 0) b -= l * __shfl_sync(0xffffffffu, b, p);
      // row q of column q + 1 is final now: the next owner fetches it before the barrier
      if (q + 1 < M && w == ((q + 1) & 3)) pc_next = __shfl_sync(0xffffffffu, v[(q + 1) >> 2], q);
      __syncthreads();
    }
  }
  // upper factor to shared memory; warp 0 back-substitutes with the kept reciprocals
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int c = 4 * k + w;
    Ush[lane][c] = v[k];
  }
  __syncthreads();
  if (w == 0) {
    double x = 0.0;
#pragma unroll
    for (int c = 31; c >= 0; --c) {
      if (c < M) {
        const double xc = __shfl_sync(0xffffffffu, b, c) * invd[c];
        if (lane == c) x = xc;
        if (lane < c) b -= Ush[lane][c] * xc;
      }
    }
    if (lane < M) Y[(size_t)i * M + lane] = x;
  }
  if (bad && lane == 0) taps_flag(status, TAPS_DEV_SINGULAR);
}

// One CTA per node i (M > 32): solve (mu_i C_A + C_B) y = g_i by LU with partial
// pivoting in shared memory, the right-hand side carried along as column M.  Per
// step p, warp 0 finds the pivot row (largest magnitude, ties to the smaller row;
// integer compares of the magnitudes' bit patterns), swaps it into place and takes the
// pivot's reciprocal; then warp w updates the rows
// r = p+1+w, p+5+w, ... (lanes over the columns c > p, coalesced) with one FMA per
// entry, T[r][c] -= l_r T[p][c], l_r = T[r][p] / T[p][p] (as a product with the
// reciprocal, seed plus refinement, formed by warp 0 for all rows at once).  The
// trailing update is FP64 FMA issue on all four SM sub-partitions (eight warps, so that
// two CTAs per SM keep four warps on each sub-partition); two barriers per step.  Back
// substitution column by column: x_r = b_r U_rr^-1 (the kept reciprocal), then every
// thread removes x_r from its rows' right-hand sides.  A zero or non-finite
// pivot is reported as TAPS_DEV_SINGULAR.
__global__ void __launch_bounds__(256) fd_small_solve_kernel(const double* __restrict__ CA,
                                                             const double* __restrict__ CB,
                                                             const double* __restrict__ mu,
                                                             const double* __restrict__ G, int M,
                                                             double* __restrict__ Y, int* status) {
  extern __shared__ double T[];   // [M][M+1]: matrix | rhs
  __shared__ double invd[TAPS_MAX_M];   // reciprocals of the pivots
  __shared__ double lmul[TAPS_MAX_M];   // the step's multipliers, by row
  __shared__ int bad;
  const int i = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nw = nt >> 5;
  const int ld = M + 1;
  const double mi = mu ? mu[i] : 0.0;
  for (int idx = tid; idx < M * M; idx += nt) {
    int r = idx / M, c = idx % M;
    T[r * ld + c] = (CA ? mi * CA[idx] : 0.0) + CB[idx];
  }
  for (int r = tid; r < M; r += nt) T[r * ld + M] = G[(size_t)i * M + r];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int p = 0; p < M; ++p) {
    if (warp == 0) {   // argmax |T[r][p]|, r >= p (ties to the smaller r), swap, reciprocal
      // compared as the bit patterns of |T[r][p]| (non-negative doubles order like
      // their bits): integer compares, off the FP64 pipe the update warps keep busy
      long long best = -1;
      int br = p;
      for (int r = p + lane; r < M; r += 32) {
        const long long a = __double_as_longlong(fabs(T[r * ld + p]));
        if (a > best) { best = a; br = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const long long ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int orr = __shfl_xor_sync(0xffffffffu, br, o);
        if (ob > best || (ob == best && orr < br)) { best = ob; br = orr; }
      }
      if (br != p)
        for (int c = p + lane; c <= M; c += 32) {
          const double t = T[p * ld + c];
          T[p * ld + c] = T[br * ld + c];
          T[br * ld + c] = t;
        }
      __syncwarp();
      const double pv = T[p * ld + p];
      const bool ok = taps_finite_nonzero(pv);
      const double inv = ok ? taps_rcp(pv) : 0.0;
      if (lane == 0) {
        invd[p] = inv;
        if (!ok) bad = 1;
      }
      // the multipliers of every row below, lanes over rows: one FP64 instruction per
      // 32 rows instead of one per row in the update warps
      for (int r = p + 1 + lane; r < M; r += 32) lmul[r] = T[r * ld + p] * inv;
    }
    __syncthreads();
    for (int r = p + 1 + warp; r < M; r += nw) {
      const double l = lmul[r];
      for (int c = p + 1 + lane; c <= M; c += 32) T[r * ld + c] = fma(-l, T[p * ld + c], T[r * ld + c]);
    }
    __syncthreads();
  }
  for (int r = M - 1; r >= 0; --r) {
    if (tid == 0) T[r * ld + M] *= invd[r];   // the kept reciprocal (0 for a bad pivot)
    __syncthreads();
    const double xr = T[r * ld + M];
    for (int k = tid; k < r; k += nt) T[k * ld + M] = fma(-T[k * ld + r], xr, T[k * ld + M]);
    __syncthreads();
  }
  for (int r = tid; r < M; r += nt) Y[(size_t)i * M + r] = T[r * ld + M];
  if (tid == 0 && bad) taps_flag(status, TAPS_DEV_SINGULAR);
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
static bool op_symmetric(int op) { return op != TAPS_OP_G; }
static bool op_mass_like(int op) { return op == TAPS_OP_M || op == TAPS_OP_W; }

// Slot choice of dim d: returns 1 with (slotA, slotB) (slotA = -1 when the dim has a
// single operator) if the dim's distinct operators form a symmetric pencil with a
// mass-like (positive definite) partner.
int taps_fd_eligible(const taps_problem* P, int d, int* slotA, int* slotB) {
  int n = P->tt.nops[d];
  if (n < 1 || n > 2) return 0;
  for (int s = 0; s < n; ++s)
    if (P->ops[d][s] >= TAPS_NUM_OPS) return 0;   // weighted operators: block elimination
  for (int s = 0; s < n; ++s)
    if (!op_symmetric(P->ops[d][s])) return 0;
  if (n == 1) {
    *slotA = -1;
    *slotB = 0;
    return 1;
  }
  int b = op_mass_like(P->ops[d][0]) ? 0 : (op_mass_like(P->ops[d][1]) ? 1 : -1);
  if (b < 0) return 0;
  *slotB = b;
  *slotA = 1 - b;
  return 1;
}

static void fd_pending_free(FdPending& T) {
  cudaFree(T.A);
  cudaFree(T.B);
  cudaFree(T.V);
  cudaFree(T.tmp);
  cudaFree(T.bt);
  cudaFree(T.dd);
  cudaFree(T.ee);
  cudaFree(T.lam);
  cudaFree(T.W);
  memset(&T, 0, sizeof(T));
}

// Cluster size of the tridiagonalisation: 16 CTAs when the device can run a 16-CTA
// cluster of the kernel (non-portable size), else the portable 8.  Both variants do the
// same arithmetic per row and per reduction, so the result does not depend on it.
template <int NC>
static bool td_cluster_ok(const void* fn, size_t smem) {
  if (NC > 8 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int maxsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (taps_allow_dyn_smem(fn, maxsm) != TAPS_OK) {
    cudaGetLastError();
    return false;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC);
  cfg.blockDim = dim3(TD_THREADS);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return clusters > 0;
}

template <int NC, typename... Args>
static cudaError_t td_launch(void (*fn)(Args...), size_t smem, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(NC);
  cfg.blockDim = dim3(TD_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = NC;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, args...);
}

// The tridiagonalisation of S (n x n in A) on one cluster: S in distributed shared
// memory when its rows fit, else in global memory.
static int td_run(double* A, double* V, double* tmp, double* bt, double* dd, double* ee, int n, int maxsm,
                  cudaStream_t s) {
  const size_t dsm16 = sizeof(double) * ((size_t)((n + 15) / 16) * n + 3 * (size_t)n);
  const size_t dsm8 = sizeof(double) * ((size_t)((n + 7) / 8) * n + 3 * (size_t)n);
  const size_t gsm = sizeof(double) * 3 * (size_t)n;
  cudaError_t ce;
  if (dsm16 + 1024 <= (size_t)maxsm && td_cluster_ok<16>((const void*)fd_tridiag_dsmem_kernel<16>, dsm16)) {
    ce = td_launch<16>(fd_tridiag_dsmem_kernel<16>, dsm16, s, (const double*)A, V, bt, dd, ee, n);
  } else if (dsm8 + 1024 <= (size_t)maxsm && td_cluster_ok<8>((const void*)fd_tridiag_dsmem_kernel<8>, dsm8)) {
    ce = td_launch<8>(fd_tridiag_dsmem_kernel<8>, dsm8, s, (const double*)A, V, bt, dd, ee, n);
  } else if (td_cluster_ok<16>((const void*)fd_tridiag_kernel<16>, gsm)) {
    ce = td_launch<16>(fd_tridiag_kernel<16>, gsm, s, A, V, tmp, bt, dd, ee, n);
  } else {
    if (!td_cluster_ok<8>((const void*)fd_tridiag_kernel<8>, gsm)) return TAPS_ERR_CUDA;
    ce = td_launch<8>(fd_tridiag_kernel<8>, gsm, s, A, V, tmp, bt, dd, ee, n);
  }
  if (ce != cudaSuccess) {
    taps_note_cuda_error(ce, "tridiagonalisation launch", __FILE__, __LINE__);
    return TAPS_ERR_CUDA;
  }
  return TAPS_OK;
}

// Enqueues the decomposition of the pencil (opA, opB) of dm on P's stream without
// waiting for it: the entry is registered at once (pending, with an event recorded
// after its last kernel) and the temporaries are returned in *T for fd_finish.  An
// entry that already exists, pending on another stream, makes P's stream wait for it.
static int fd_enqueue(taps_problem* P, taps_dim* dm, int opA, int opB, FdEntry** out, FdPending* T) {
  memset(T, 0, sizeof(*T));
  for (int k = 0; k < dm->nfd; ++k)
    if (dm->fd[k].opA == opA && dm->fd[k].opB == opB) {
      *out = &dm->fd[k];
      if (dm->fd[k].pending && dm->fd[k].done) TAPS_CUDA(cudaStreamWaitEvent(P->stream, dm->fd[k].done, 0));
      return dm->fd[k].status;
    }
  if (dm->nfd >= 4) return TAPS_ERR_INVALID_ARG;
  FdEntry& E = dm->fd[dm->nfd];
  memset(&E, 0, sizeof(E));
  E.opA = opA;
  E.opB = opB;
  int n = dm->nf;
  size_t nn = (size_t)n * n;
  cudaStream_t s = P->stream;
  const int hasA = opA >= 0 ? 1 : 0;
  int st = TAPS_OK;
  T->E = &E;
  T->P = P;
  do {
    // the back-transform keeps one column per warp in shared memory (n <= 6144); the
    // tridiagonalisation stages three vectors (3n doubles)
    if (sizeof(double) * (size_t)n > 48 * 1024) { st = TAPS_ERR_INVALID_ARG; break; }
    int maxsm_optin = 0;
    {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&maxsm_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    }
    if ((st = taps_alloc((void**)&E.Phi, sizeof(double) * nn)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&E.PhiT, sizeof(double) * nn)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&E.mu, sizeof(double) * n)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->A, sizeof(double) * nn)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->B, sizeof(double) * nn)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->V, sizeof(double) * nn)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->tmp, sizeof(double) * 2 * n)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->bt, sizeof(double) * n)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->dd, sizeof(double) * n)) != TAPS_OK) break;
    if ((st = taps_alloc((void**)&T->ee, sizeof(double) * n)) != TAPS_OK) break;
    if (hasA) {
      if ((st = taps_alloc((void**)&T->lam, sizeof(double) * n)) != TAPS_OK) break;
      if ((st = taps_alloc((void**)&T->W, sizeof(double) * 5 * nn)) != TAPS_OK) break;
    }
    double *A = T->A, *B = T->B, *V = T->V, *W = T->W, *lam = T->lam;
    const size_t bsz = (size_t)n * dm->nb;
    const double* bandA = hasA ? dm->d_band + (size_t)opA * bsz : nullptr;
    const double* bandB = dm->d_band + (size_t)opB * bsz;
    int tk = prof_begin(P, TAPS_PROF_OTHER);
    fd_dense_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(bandA, bandB, n, dm->hb, A, B);
    if (cudaMemsetAsync(V, 0, sizeof(double) * nn, s) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
    // banded Cholesky and S (one CTA), then the tridiagonalisation (one cluster)
    fd_setup_kernel<<<1, FD_THREADS, 0, s>>>(B, n, dm->hb, P->d_status);
    if (hasA) {
      // S = L^{-1} A L^{-T}: X = L^{-1} A into V, S^T = L^{-1} X^T into W, symmetrised into A
      fd_lsolve_kernel<<<(n + 31) / 32, 32, 0, s>>>(B, A, n, dm->hb, 0, V);
      fd_lsolve_kernel<<<(n + 31) / 32, 32, 0, s>>>(B, V, n, dm->hb, 1, W);
      fd_symmetrize_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, s>>>(W, n, A);
      if (cudaMemsetAsync(V, 0, sizeof(double) * nn, s) != cudaSuccess) { st = TAPS_ERR_CUDA; break; }
      if ((st = td_run(A, V, T->tmp, T->bt, T->dd, T->ee, n, maxsm_optin, s)) != TAPS_OK) break;
      // eigenvalues (warp each), eigenvectors (thread each), back-transform (warp each),
      // all into A, which the tridiagonalisation no longer needs
      // two warps per CTA: the warps' FP64 chains spread over the SMs' sub-partitions
      fd_bisect_kernel<<<(unsigned)((32LL * n + 63) / 64), 64, 0, s>>>(T->dd, T->ee, n, lam);
      // one thread per eigenvector in 32-thread CTAs: the chains spread over the SMs
      fd_invit_kernel<<<(n + 31) / 32, 32, 0, s>>>(T->dd, T->ee, lam, n, A, W);
      // symmetric orthogonalisation: E in W, the corrected vectors back into A
      const unsigned gnn = (unsigned)((nn + 255) / 256);
      fd_gram_minus_identity_kernel<<<gnn, 256, 0, s>>>(A, n, W);
      fd_orth_update_kernel<<<gnn, 256, 0, s>>>(A, W, n, W + nn);
      if (cudaMemcpyAsync(A, W + nn, sizeof(double) * nn, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
        st = TAPS_ERR_CUDA;
        break;
      }
      const int wpc = std::max(1, std::min(8, (int)(48 * 1024 / (sizeof(double) * (size_t)n))));
      fd_backtransform_kernel<<<(n + wpc - 1) / wpc, 32 * wpc, sizeof(double) * (size_t)n * wpc, s>>>(
          V, T->bt, n, A);
    }
    fd_phi_kernel<<<(n + 31) / 32, 32, 0, s>>>(B, hasA ? A : nullptr, hasA ? lam : nullptr, n, dm->hb, E.Phi,
                                                  E.PhiT, E.mu, P->d_status);
    prof_end(P, TAPS_PROF_OTHER, tk, (10.0 / 3.0) * (double)nn * n, 8.0 * 4.0 * nn);
    cudaError_t ce = cudaGetLastError();
    if (ce != cudaSuccess) {
      taps_note_cuda_error(ce, "pencil decomposition", __FILE__, __LINE__);
      st = TAPS_ERR_CUDA;
      break;
    }
    if (cudaEventCreateWithFlags(&E.done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(E.done, s) != cudaSuccess) {
      st = TAPS_ERR_CUDA;
      break;
    }
  } while (0);
  E.status = st;
  E.pending = (st == TAPS_OK) ? 1 : 0;
  dm->nfd++;
  *out = &E;
  if (st != TAPS_OK) fd_pending_free(*T);
  return st;
}

// Waits for a decomposition enqueued by fd_enqueue, reads its problem's device status
// into the entry and frees the temporaries.
static int fd_finish(FdPending& T) {
  if (!T.E) return TAPS_OK;
  int st = taps_check_status(T.P->d_status, T.P->stream);
  if (T.E->status == TAPS_OK) T.E->status = st;
  T.E->pending = 0;
  if (T.E->done) {
    cudaEventDestroy(T.E->done);
    T.E->done = nullptr;
  }
  fd_pending_free(T);
  return st;
}

static int fd_prepare(taps_problem* P, int d, taps_dim* dm, int opA, int opB, FdEntry** out) {
  (void)d;
  FdPending T;
  int st = fd_enqueue(P, dm, opA, opB, out, &T);
  if (st != TAPS_OK) return st;
  return fd_finish(T);
}

// Reduced solve of dim d by fast diagonalisation, coefficients in P->d_C / P->d_c.
int taps_fd_solve(taps_problem* P, taps_factors* U, int d, int precision) {
  int slotA, slotB;
  if (!taps_fd_eligible(P, d, &slotA, &slotB)) return TAPS_ERR_INVALID_ARG;
  taps_dim* dm = P->dims[d];
  FdEntry* E = nullptr;
  int opA = slotA >= 0 ? P->ops[d][slotA] : -1;
  TAPS_TRY(fd_prepare(P, d, dm, opA, P->ops[d][slotB], &E));
  if (!P->d_pq[d]) return TAPS_ERR_INVALID_ARG;   // taps_fd_prepare_all comes first
  const int n = dm->nf, M = U->M;
  const size_t MM = (size_t)M * M;
  cudaStream_t s = P->stream;
  const int nM = n * M;
  double* G = P->d_Y;
  double* Y = P->d_Y + (size_t)n * M;
  int tk = prof_begin(P, TAPS_PROF_FASTDIAG);
  const double* CA = slotA >= 0 ? P->d_C + (size_t)slotA * MM : nullptr;
  const double* CB = P->d_C + (size_t)slotB * MM;
  int launches = 2;
  if (M <= 32 && precision != TAPS_MIXED) {
    TAPS_CUDA(taps_launch_pdl(fd_small_solve_quad_kernel, dim3(n), dim3(128), 0, s, CA, CB,
                              slotA >= 0 ? (const double*)E->mu : nullptr, (const double*)P->d_pq[d],
                              (const double*)P->d_c, P->Rf, n, M, Y, P->d_status));
  } else {
    fd_rhs_kernel<<<(nM + 255) / 256, 256, 0, s>>>(P->d_pq[d], P->d_c, P->Rf, n, M, G);
    if (M <= 32)
      fd_small_solve_warp_kernel<<<n, 32, 0, s>>>(CA, CB, slotA >= 0 ? E->mu : nullptr, G, n, M, Y,
                                                  P->d_status, 1);
    else {
      // M (M + 1) doubles exceed the default 48 KB from M = 78 on: allow up to M = 128
      static bool smem_ok = false;
      if (!smem_ok) {
        int dev = 0, maxsm = 0;
        TAPS_CUDA(cudaGetDevice(&dev));
        TAPS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        TAPS_TRY(taps_allow_dyn_smem((const void*)fd_small_solve_kernel, maxsm));
        smem_ok = true;
      }
      fd_small_solve_kernel<<<n, 256, sizeof(double) * (size_t)M * (M + 1), s>>>(
          CA, CB, slotA >= 0 ? E->mu : nullptr, G, M, Y, P->d_status);
    }
    ++launches;
  }
  P->prof->launches[TAPS_PROF_FASTDIAG] += launches - 2;
  prof_end(P, TAPS_PROF_FASTDIAG, tk, 2.0 * P->Rf * nM + n * ((2.0 / 3.0) * M * MM + 2.0 * MM),
           8.0 * ((double)P->Rf * n + 2.0 * MM + (double)nM));
  // back to the nodal basis; the previous factor goes to d_Uold for the change norm
  tk = prof_begin(P, TAPS_PROF_FD_TRANSFORM);
  TAPS_CUDA(taps_launch_pdl(fd_rowgemm_kernel, dim3(n), dim3(RG_WARPS * 32), 0, s, (const double*)E->Phi,
                            (const double*)Y, n, M, U->d_U[d], 1, P->d_Uold));
  prof_end(P, TAPS_PROF_FD_TRANSFORM, tk, 2.0 * (double)n * n * M, 8.0 * ((double)n * n + 3.0 * nM));
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

// The cached (or newly made) decomposition of the pencil (opA, opB) of dim d.
int taps_fd_lookup(taps_problem* P, int d, int opA, int opB, const FdEntry** out) {
  FdEntry* E = nullptr;
  TAPS_TRY(fd_prepare(P, d, P->dims[d], opA, opB, &E));
  *out = E;
  return TAPS_OK;
}

// Out = Phi Y in the factor layout (Y n x M row-major), the previous factor into Save.
int taps_fd_to_nodal(taps_problem* P, const FdEntry* E, const double* Y, int n, int M, double* Out, double* Save) {
  int tk = prof_begin(P, TAPS_PROF_FD_TRANSFORM);
  TAPS_CUDA(taps_launch_pdl(fd_rowgemm_kernel, dim3(n), dim3(RG_WARPS * 32), 0, P->stream, (const double*)E->Phi,
                            Y, n, M, Out, 1, Save));
  prof_end(P, TAPS_PROF_FD_TRANSFORM, tk, 2.0 * (double)n * n * M, 8.0 * ((double)n * n + 3.0 * (double)n * M));
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

// Pencil decompositions of every eligible dim, done before any capture (they
// allocate and synchronise).  The enqueue half launches them on P's stream and keeps
// their temporaries in *pend; the finish half waits, checks and frees.  Batches
// enqueue many problems (each on its own stream) before finishing any, so the
// decompositions of different instances run concurrently.
int taps_fd_prepare_enqueue(taps_problem* P, int solver, int M, std::vector<FdPending>* pend) {
  if (solver != TAPS_SOLVER_FASTDIAG && solver != TAPS_SOLVER_MODEDIAG) return TAPS_OK;
  for (int d = 0; d < P->D; ++d) {
    int sa, sb;
    const int route = taps_dim_route(P, d, solver, M);
    if (route == TAPS_ROUTE_FDW) {
      int s0, s1, nb;
      taps_fdw_eligible(P, d, M, &sa, &sb, &s0, &s1, &nb);
    } else if (route != TAPS_ROUTE_FD || !taps_fd_eligible(P, d, &sa, &sb)) {
      continue;
    }
    FdEntry* E = nullptr;
    FdPending T;
    TAPS_TRY(fd_enqueue(P, P->dims[d], sa >= 0 ? P->ops[d][sa] : -1, P->ops[d][sb], &E, &T));
    if (T.E) pend->push_back(T);
    if (!P->d_pq[d]) {   // the problem's source vectors in the pencil's eigenbasis
      const int n = P->dims[d]->nf;
      const long long tot = (long long)n * P->Rf;
      TAPS_TRY(taps_alloc((void**)&P->d_pq[d], sizeof(double) * (size_t)std::max(tot, 1LL)));
      if (tot > 0)
        fd_pq_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, P->stream>>>(E->PhiT, P->d_q[d], n, P->Rf,
                                                                           P->d_pq[d]);
      TAPS_CUDA(cudaGetLastError());
    }
  }
  return TAPS_OK;
}

int taps_fd_prepare_finish(std::vector<FdPending>* pend) {
  int st = TAPS_OK;
  for (auto& T : *pend) {
    int s2 = fd_finish(T);
    if (st == TAPS_OK) st = s2;
  }
  pend->clear();
  return st;
}

int taps_fd_prepare_all(taps_problem* P, int solver, int M) {
  std::vector<FdPending> pend;
  int st = taps_fd_prepare_enqueue(P, solver, M, &pend);
  int s2 = taps_fd_prepare_finish(&pend);
  return st != TAPS_OK ? st : s2;
}

void taps_fd_release(taps_dim* dm) {
  for (int k = 0; k < dm->nfd; ++k) {
    cudaFree(dm->fd[k].Phi);
    cudaFree(dm->fd[k].PhiT);
    cudaFree(dm->fd[k].mu);
    if (dm->fd[k].done) cudaEventDestroy(dm->fd[k].done);
  }
  dm->nfd = 0;
}

// ---------------------------------------------------------------------------------
// The small solves' reciprocal on a device array (for checking it against IEEE
// division).
// ---------------------------------------------------------------------------------
__global__ void rcp_kernel(const double* __restrict__ x, double* __restrict__ y, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = taps_rcp(x[i]);
}

extern "C" int taps_util_rcp(const double* x_dev, double* y_dev, long long n, void* stream) {
  if (n < 0 || (n > 0 && (!x_dev || !y_dev))) return TAPS_ERR_INVALID_ARG;
  if (n == 0) return TAPS_OK;
  rcp_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(x_dev, y_dev, n);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

// ---------------------------------------------------------------------------------
// The library's bounded grid barrier with a short poll limit, for its failure test:
// `ctas` CTAs meet at a barrier that expects ctas + missing arrivals, twice.  With
// missing > 0 every wait runs out after `limit` polls, records TAPS_DEV_TIMEOUT and the
// kernel returns; the host reads the status.  Nothing waits without a bound.
// ---------------------------------------------------------------------------------
__global__ void barrier_test_kernel(unsigned* bar, int* status, unsigned expected, long long limit) {
  grid_barrier(bar, status, expected, limit);
  grid_barrier(bar, status, expected, limit);
}

extern "C" int taps_util_barrier_test(int ctas, int missing, long long poll_limit, void* stream) {
  if (ctas < 1 || ctas > 64 || missing < 0 || missing > 64 || poll_limit < 1 || poll_limit > (1ll << 26))
    return TAPS_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* bar = nullptr;
  int* status = nullptr;
  TAPS_TRY(taps_alloc((void**)&bar, 2 * sizeof(unsigned)));
  if (taps_alloc((void**)&status, sizeof(int)) != TAPS_OK) {
    cudaFree(bar);
    return TAPS_ERR_OOM;
  }
  int st = TAPS_OK;
  if (cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), s) != cudaSuccess ||
      cudaMemsetAsync(status, 0, sizeof(int), s) != cudaSuccess) {
    st = TAPS_ERR_CUDA;
  } else {
    barrier_test_kernel<<<ctas, 32, 0, s>>>(bar, status, (unsigned)(ctas + missing), poll_limit);
    if (cudaGetLastError() != cudaSuccess) st = TAPS_ERR_CUDA;
    else st = taps_check_status(status, s);
  }
  cudaStreamSynchronize(s);
  cudaFree(bar);
  cudaFree(status);
  return st;
}
