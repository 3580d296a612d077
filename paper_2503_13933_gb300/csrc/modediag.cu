// Reduced solve by diagonalisation on the mode side (Sec. 2.6).
//
// The dim-d system of Eq. 43 is the Sylvester form  Op_X U C_X^T + Op_Y U C_Y^T = F
// whenever the dim has two distinct operators.  If every other dim's operators are
// symmetric, every Gram of the other dims is symmetric and so are C_X and C_Y (Hadamard
// products and sums of symmetric matrices).  With the generalised eigenpairs of the
// M x M pencil,  C_Y w_j = lam_j C_X w_j  (W^T C_X W = I, W^T C_Y W = diag(lam)),
// the substitution U = Z W^T splits the system into M independent banded n_d x n_d
// systems  (Op_X + lam_j Op_Y) z_j = (F W)_j.  The cost per solve is the paper's
// O(M^3 + M^2 n_d + C_c(n_d)): the eigenproblem, two n_d x M x M transforms and M
// banded eliminations; no n_d x n_d decomposition is ever formed.  This is the route
// for time dims (G and M: the time derivative makes the node-side pencil
// nonsymmetric, while the coefficients stay symmetric).
//
//   md_eig_kernel    one CTA: (in the dim's previous basis P, when it has one)
//                    Cholesky C_X = L L^T, S = L^-1 C_Y L^-T, cyclic Jacobi
//                    S = Q diag(lam) Q^T, W = P L^-T Q, and Wc_r = W^T c_r for the
//                    right-hand side F W = sum_r q_r (W^T c_r)^T.
//   md_band_kernel   thread j: Gaussian elimination without pivoting of the banded
//                    Op_X + lam_j Op_Y (half-bandwidth HB) with the active window in
//                    registers, then back substitution; Z is n_d x M row-major.
//   md_out_kernel    U = Z W^T into the factor layout, the old factor into Save.
//
// The eliminations need no pivoting: with X the mass-like operator (symmetric
// positive definite) and lam_j >= 0, the symmetric part of Op_X + lam_j Op_Y is
// positive definite (the time-derivative matrix with the initial node removed has a
// positive semidefinite symmetric part).  A zero or non-finite pivot, or a C_X that is
// indefinite beyond rounding, is reported as TAPS_DEV_SINGULAR.
#include <string.h>

#include <algorithm>

#include "taps_internal.cuh"

#define MD_THREADS 128
#define MD_MAX_HB 5
#define MD_MAX_SWEEPS 24

// C = A B, A^T B or A B^T for M x M shared-memory matrices (all threads).
__device__ __forceinline__ void md_mm(double (*C)[33], const double (*A)[33], const double (*B)[33], int M,
                                      bool transA) {
  for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
    const int i = idx / M, j = idx % M;
    double s = 0.0;
    if (transA)
      for (int k = 0; k < M; ++k) s += A[k][i] * B[k][j];
    else
      for (int k = 0; k < M; ++k) s += A[i][k] * B[k][j];
    C[i][j] = s;
  }
}

// Wp / Wout: the dim's basis from its previous solve (valid when *wM == M) and the
// new one, M x M row-major, in place.  A valid previous basis P (P^T C_X P ~ I,
// P^T C_Y P ~ diagonal as the ALS converges) is applied first: the pencil
// (P^T C_Y P, P^T C_X P) is diagonalised instead, which the Jacobi sweeps finish in a
// few sweeps, and W = P W_inner.
__global__ void __launch_bounds__(MD_THREADS) md_eig_kernel(const double* __restrict__ CX,
                                                            const double* __restrict__ CY,
                                                            const double* __restrict__ c, int Rf, int M,
                                                            double* __restrict__ Wio, int* __restrict__ wM,
                                                            double* __restrict__ lam, double* __restrict__ cw,
                                                            int* status) {
  __shared__ double L[32][33], S[32][33], V[32][33], T[32][33], Pw[32][33];
  __shared__ double linv[32];
  __shared__ double rc[16], rs[16];
  __shared__ int rp[16], rq[16];
  __shared__ int rotated, failed;
  const int tid = threadIdx.x, nt = blockDim.x;
  const bool warm = (*wM == M);
  if (tid == 0) failed = 0;
  // symmetrised coefficients (exactly symmetric in exact arithmetic)
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    L[i][j] = 0.5 * (CX[i * M + j] + CX[j * M + i]);
    S[i][j] = CY ? 0.5 * (CY[i * M + j] + CY[j * M + i]) : 0.0;   // no Y: S = 0, lam = 0
    Pw[i][j] = warm ? Wio[idx] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  if (warm) {   // L <- P^T C_X P, S <- P^T C_Y P
    md_mm(T, L, Pw, M, false);
    __syncthreads();
    md_mm(L, Pw, T, M, true);
    __syncthreads();
    md_mm(T, S, Pw, M, false);
    __syncthreads();
    md_mm(S, Pw, T, M, true);
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      if (i < j) {
        const double a = 0.5 * (L[i][j] + L[j][i]), b = 0.5 * (S[i][j] + S[j][i]);
        L[i][j] = a;
        L[j][i] = a;
        S[i][j] = b;
        S[j][i] = b;
      }
    }
    __syncthreads();
  }
  // Cholesky of the (transformed) C_X = L L^T (lower triangle of L).  C_X is positive
  // semidefinite by construction (Hadamard products and sums of Grams); with nearly
  // dependent modes its pivots can round to zero or slightly below, and such a pivot
  // is raised to 64 eps max_k C_kk (the pencil is perturbed at the rounding level of
  // its own entries, in that direction only).  A clearly negative pivot (an indefinite
  // C_X) or a non-finite one is an error.
  double dmax = 0.0;
  for (int k = 0; k < M; ++k) dmax = fmax(dmax, fabs(L[k][k]));
  const double floor_piv = 64.0 * 1.1102230246251565e-16 * dmax;
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      double piv = L[k][k];
      if (!isfinite(piv) || !(dmax > 0.0) || !isfinite(dmax) || piv < -1e-8 * dmax) {
        taps_flag(status, TAPS_DEV_SINGULAR);
        failed = 1;
        piv = 1.0;
      } else if (piv < floor_piv) {
        piv = floor_piv;
      }
      const double r = sqrt(piv);
      L[k][k] = r;
      linv[k] = taps_rcp(r);
    }
    __syncthreads();
    const double il = linv[k];
    for (int i = k + 1 + tid; i < M; i += nt) L[i][k] *= il;
    __syncthreads();
    const int w = M - k - 1;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int i = k + 1 + idx / w, j = k + 1 + idx % w;
      if (j <= i) L[i][j] -= L[i][k] * L[j][k];
    }
    __syncthreads();
  }
  // X = L^-1 C_Y into V (thread per column), then S = L^-1 X^T (thread per column)
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = S[i][col];
      for (int j = 0; j < i; ++j) s -= L[i][j] * V[j][col];
      V[i][col] = s * linv[i];
    }
  }
  __syncthreads();
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = V[col][i];
      for (int j = 0; j < i; ++j) s -= L[i][j] * S[j][col];
      S[i][col] = s * linv[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    if (i < j) {
      const double a = 0.5 * (S[i][j] + S[j][i]);
      S[i][j] = a;
      S[j][i] = a;
    }
    V[i][j] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  // cyclic Jacobi, round-robin pairing: N = M rounded up to even players, N - 1
  // rounds of N / 2 disjoint pairs per sweep; a pair with the padding player idles
  const int N = M + (M & 1), half = N / 2;
  for (int sw = 0; sw < MD_MAX_SWEEPS && M > 1; ++sw) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < N - 1; ++r) {
      if (tid < half) {
        int a, b;
        if (tid == 0) {
          a = r;
          b = N - 1;
        } else {
          a = (r + tid) % (N - 1);
          b = (r - tid + N - 1) % (N - 1);
        }
        const int p = min(a, b), q = max(a, b);
        double cs = 1.0, sn = 0.0;
        if (q < M) {
          const double apq = S[p][q], app = S[p][p], aqq = S[q][q];
          // rotate unless a_pq is negligible against the diagonal (relative accuracy)
          if (fabs(apq) > 1.1102230246251565e-16 * sqrt(fabs(app * aqq)) && fabs(apq) > 1e-300) {
            const double th = (aqq - app) * taps_rcp(2.0 * apq);
            double t;
            if (fabs(th) > 1e150) {
              t = 0.5 * taps_rcp(th);
            } else {
              t = taps_rcp(fabs(th) + sqrt(th * th + 1.0));
              if (th < 0.0) t = -t;
            }
            cs = taps_rcp(sqrt(t * t + 1.0));
            sn = t * cs;
            rotated = 1;
          }
        }
        rc[tid] = cs;
        rs[tid] = sn;
        rp[tid] = p;
        rq[tid] = q;
      }
      __syncthreads();
      // columns p, q of S and V: S <- S J, V <- V J
      for (int idx = tid; idx < half * M; idx += nt) {
        const int k = idx / M, i = idx % M;
        const double sn = rs[k];
        if (sn != 0.0) {
          const double cs = rc[k];
          const int p = rp[k], q = rq[k];
          const double sp = S[i][p], sq = S[i][q];
          S[i][p] = cs * sp - sn * sq;
          S[i][q] = sn * sp + cs * sq;
          const double vp = V[i][p], vq = V[i][q];
          V[i][p] = cs * vp - sn * vq;
          V[i][q] = sn * vp + cs * vq;
        }
      }
      __syncthreads();
      // rows p, q of S: S <- J^T S
      for (int idx = tid; idx < half * M; idx += nt) {
        const int k = idx / M, j = idx % M;
        const double sn = rs[k];
        if (sn != 0.0) {
          const double cs = rc[k];
          const int p = rp[k], q = rq[k];
          const double sp = S[p][j], sq = S[q][j];
          S[p][j] = cs * sp - sn * sq;
          S[q][j] = sn * sp + cs * sq;
        }
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // W_inner = L^-T Q in place of V (thread per column, bottom row first)
  if (tid < M) {
    const int col = tid;
    for (int i = M - 1; i >= 0; --i) {
      double s = V[i][col];
      for (int j = i + 1; j < M; ++j) s -= L[j][i] * V[j][col];
      V[i][col] = s * linv[i];
    }
  }
  __syncthreads();
  // W = P W_inner
  md_mm(T, Pw, V, M, false);
  __syncthreads();
  bool finite = true;
  for (int idx = tid; idx < M * M; idx += nt) {
    const double w = T[idx / M][idx % M];
    finite &= isfinite(w);
    Wio[idx] = w;
  }
  if (!finite) failed = 1;
  for (int j = tid; j < M; j += nt) lam[j] = S[j][j];
  for (int idx = tid; idx < Rf * M; idx += nt) {
    const int r = idx / M, j = idx % M;
    double s = 0.0;
    for (int m = 0; m < M; ++m) s += c[r * M + m] * T[m][j];
    cw[idx] = s;
  }
  __syncthreads();
  // the basis seeds the next solve of this dim only if it is sound
  if (tid == 0) *wM = failed ? 0 : M;
}

// Element (row, col) of Op_X + lam Op_Y from the [n][2HB+1] bands; zero outside.
template <int HB>
__device__ __forceinline__ double md_elem(const double* __restrict__ bx, const double* __restrict__ by,
                                          double lam, int n, int row, int col) {
  const int k = col - row + HB;
  if (row >= n || col >= n || k < 0 || k > 2 * HB) return 0.0;
  const size_t o = (size_t)row * (2 * HB + 1) + k;
  return bx[o] + lam * by[o];
}

// Right-hand side entry (F W)[row][j] = sum_r q_r[row] Wc_r[j].
__device__ __forceinline__ double md_rhs(const double* __restrict__ q, const double* __restrict__ cw, int Rf,
                                         int n, int M, int row, int j) {
  if (row >= n) return 0.0;
  double s = 0.0;
  for (int r = 0; r < Rf; ++r) s += q[(size_t)r * n + row] * cw[r * M + j];
  return s;
}

// Thread j < M solves (Op_X + lam_j Op_Y) z_j = (F W)_j.  Forward elimination keeps
// rows i .. i+HB of the active matrix in registers (row i+r holds columns i .. i+r+HB;
// Gaussian elimination of a band matrix without pivoting creates no fill outside the
// band) and stores, per step, the pivot row scaled by the pivot's reciprocal; back
// substitution walks the stored rows upwards.  Stored rows: scratch[i][c][j],
// c = 0 (scaled right-hand side), 1..HB (scaled superdiagonal entries).
// Raw band row `row` of X and Y, columns c0 .. c0 + 2HB (zero outside the matrix),
// and its right-hand side entry: loaded two elimination steps before the row enters
// the window, so that the loads' latency stays off the pivot chain.
template <int HB>
__device__ __forceinline__ void md_stage(const double* __restrict__ bx, const double* __restrict__ by,
                                         const double* __restrict__ q, const double* __restrict__ cw, int Rf,
                                         int n, int M, int j, int row, int c0, double* x, double* y, double& r) {
  constexpr int W2 = 2 * HB + 1;
  const bool in = row < n;
  const size_t o = (size_t)(in ? row : 0) * W2;
#pragma unroll
  for (int c = 0; c < W2; ++c) {
    const bool ok = in && (c0 + c) < n && (c0 + c) >= 0 && (c0 + c - row + HB) >= 0 && (c0 + c - row + HB) < W2;
    const int k = c0 + c - row + HB;
    x[c] = ok ? bx[o + k] : 0.0;
    y[c] = ok ? by[o + k] : 0.0;
  }
  r = md_rhs(q, cw, Rf, n, M, row, j);
}

// Thread j < M solves (Op_X + lam_j Op_Y) z_j = (F W)_j.  Forward elimination keeps
// rows i .. i+HB of the active matrix in registers (row i+r holds columns i .. i+r+HB;
// Gaussian elimination of a band matrix without pivoting creates no fill outside the
// band) and stores, per step, the pivot row scaled by the pivot's reciprocal; back
// substitution walks the stored rows upwards.  Stored rows: scratch[i][c][j],
// c = 0 (scaled right-hand side), 1..HB (scaled superdiagonal entries).
template <int HB>
__global__ void __launch_bounds__(32) md_band_kernel(const double* __restrict__ bx, const double* __restrict__ by,
                                                     const double* __restrict__ lam, const double* __restrict__ q,
                                                     const double* __restrict__ cw, int Rf, int n, int M,
                                                     double* __restrict__ scratch, double* __restrict__ Z,
                                                     int* status) {
  const int j = threadIdx.x;
  if (j >= M) return;
  const double lj = lam[j];
  constexpr int W2 = 2 * HB + 1;
  double A[HB + 1][W2];
  double b[HB + 1];
#pragma unroll
  for (int r = 0; r <= HB; ++r) {
#pragma unroll
    for (int c = 0; c < W2; ++c) A[r][c] = (c <= r + HB) ? md_elem<HB>(bx, by, lj, n, r, c) : 0.0;
    b[r] = md_rhs(q, cw, Rf, n, M, r, j);
  }
  // the rows entering at the ends of steps 0 and 1
  double x1[W2], y1[W2], r1, x2[W2], y2[W2], r2;
  md_stage<HB>(bx, by, q, cw, Rf, n, M, j, 1 + HB, 1, x1, y1, r1);
  md_stage<HB>(bx, by, q, cw, Rf, n, M, j, 2 + HB, 2, x2, y2, r2);
  bool bad = false;
  for (int i = 0; i < n; ++i) {
    const double piv = A[0][0];
    const bool ok = fabs(piv) > 0.0 && isfinite(piv);
    bad |= !ok;
    const double inv = ok ? taps_rcp(piv) : 0.0;
    double l[HB + 1];
#pragma unroll
    for (int r = 1; r <= HB; ++r) l[r] = A[r][0] * inv;
#pragma unroll
    for (int r = 1; r <= HB; ++r) {
#pragma unroll
      for (int c = 1; c <= HB; ++c) A[r][c] -= l[r] * A[0][c];
      b[r] -= l[r] * b[0];
    }
    double* out = scratch + (size_t)i * (HB + 1) * M + j;
    out[0] = b[0] * inv;
#pragma unroll
    for (int c = 1; c <= HB; ++c) out[(size_t)c * M] = A[0][c] * inv;
    // slide the window down one row and one column; row i+HB+1 enters
#pragma unroll
    for (int r = 0; r < HB; ++r) {
#pragma unroll
      for (int c = 0; c < W2 - 1; ++c) A[r][c] = A[r + 1][c + 1];
      A[r][W2 - 1] = 0.0;
      b[r] = b[r + 1];
    }
#pragma unroll
    for (int c = 0; c < W2; ++c) {
      A[HB][c] = fma(lj, y1[c], x1[c]);
      x1[c] = x2[c];
      y1[c] = y2[c];
    }
    b[HB] = r1;
    r1 = r2;
    md_stage<HB>(bx, by, q, cw, Rf, n, M, j, i + 3 + HB, i + 3, x2, y2, r2);
  }
  if (bad) taps_flag(status, TAPS_DEV_SINGULAR);
  // back substitution: z_i = y_i - sum_c u_ic z_{i+c}; zr[c] = z_{i+c}; the stored
  // rows are loaded two steps ahead
  double zr[HB + 1];
#pragma unroll
  for (int c = 0; c <= HB; ++c) zr[c] = 0.0;
  double u1[HB + 1], u2[HB + 1];
#pragma unroll
  for (int c = 0; c <= HB; ++c) {
    u1[c] = n - 1 >= 0 ? scratch[(size_t)(n - 1) * (HB + 1) * M + (size_t)c * M + j] : 0.0;
    u2[c] = n - 2 >= 0 ? scratch[(size_t)(n - 2) * (HB + 1) * M + (size_t)c * M + j] : 0.0;
  }
  for (int i = n - 1; i >= 0; --i) {
    // the terms of z_{i+2} .. z_{i+HB} first: only the last FMA waits for z_{i+1}
    double s = u1[0];
#pragma unroll
    for (int c = HB; c >= 2; --c) s -= u1[c] * zr[c];
    s -= u1[1] * zr[1];
#pragma unroll
    for (int c = HB; c >= 2; --c) zr[c] = zr[c - 1];
    zr[1] = s;
    Z[(size_t)i * M + j] = s;
    const int nx = i - 2;
#pragma unroll
    for (int c = 0; c <= HB; ++c) {
      u1[c] = u2[c];
      u2[c] = nx >= 0 ? scratch[(size_t)nx * (HB + 1) * M + (size_t)c * M + j] : 0.0;
    }
  }
}

// U[m][i] (factor layout, column m contiguous) = sum_j Z[i][j] W[m][j]; the previous
// factor goes to Save first (same thread, same element).
__global__ void md_out_kernel(const double* __restrict__ Z, const double* __restrict__ Wm, int n, int M,
                              double* __restrict__ U, double* __restrict__ Save) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * M) return;
  const int m = (int)(idx / n), i = (int)(idx % n);
  const double* z = Z + (size_t)i * M;
  const double* w = Wm + (size_t)m * M;
  double s = 0.0;
  for (int k = 0; k < M; ++k) s += z[k] * w[k];
  Save[idx] = U[idx];
  U[idx] = s;
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
static bool md_op_symmetric(int op) { return op != TAPS_OP_G; }
static bool md_op_mass_like(int op) { return op == TAPS_OP_M || op == TAPS_OP_W; }

int taps_md_eligible(const taps_problem* P, int d, int M, int* slotX, int* slotY) {
  const int nops = P->tt.nops[d];
  if (nops < 1 || nops > 2 || M < 1 || M > 32) return 0;
  const int hb = P->dims[d]->hb;
  if (hb < 1 || hb > MD_MAX_HB) return 0;
  for (int e = 0; e < P->D; ++e) {
    if (e == d) continue;
    for (int s = 0; s < P->tt.nops[e]; ++s)
      if (!md_op_symmetric(P->ops[e][s])) return 0;
  }
  if (nops == 1) {   // Op U C^T = F: W = L^-T, lam = 0, banded solves with Op
    *slotX = 0;
    *slotY = -1;
    return 1;
  }
  const int x = md_op_mass_like(P->ops[d][0]) ? 0 : (md_op_mass_like(P->ops[d][1]) ? 1 : 0);
  *slotX = x;
  *slotY = 1 - x;
  return 1;
}

int taps_dim_route(const taps_problem* P, int d, int solver, int M) {
  int a, b;
  if (solver == TAPS_SOLVER_MODEDIAG) {
    if (taps_md_eligible(P, d, M, &a, &b)) return TAPS_ROUTE_MD;
    if (taps_fd_eligible(P, d, &a, &b)) return TAPS_ROUTE_FD;
    return TAPS_ROUTE_LU;
  }
  if (solver == TAPS_SOLVER_FASTDIAG) {
    if (taps_fd_eligible(P, d, &a, &b)) return TAPS_ROUTE_FD;
    if (taps_md_eligible(P, d, M, &a, &b) && P->tt.nops[d] == 2) return TAPS_ROUTE_MD;
  }
  return TAPS_ROUTE_LU;
}

// [TAPS_MAX_DIMS][M][M] bases, TAPS_MAX_DIMS ints (one double each), lam [M], W^T c
// [Rf][M], Z [nf_max][M], eliminated rows [nf_max][MD_MAX_HB + 1][M].  The caller
// zeroes it (no valid basis).
size_t taps_md_scratch_doubles(int nf_max, int M, int Rf) {
  return (size_t)TAPS_MAX_DIMS * M * M + TAPS_MAX_DIMS + M + (size_t)Rf * M + (size_t)nf_max * M +
         (size_t)nf_max * (MD_MAX_HB + 1) * M;
}

// Forgets every dim's stored basis (the next solves start cold).  Called when a sweep
// call starts, so that the same factors always give the same rounding.
int taps_md_reset(taps_problem* P) {
  if (!P->d_md || P->ws_M < 1) return TAPS_OK;
  TAPS_CUDA(cudaMemsetAsync(P->d_md + (size_t)TAPS_MAX_DIMS * P->ws_M * P->ws_M, 0, sizeof(int) * TAPS_MAX_DIMS,
                            P->stream));
  return TAPS_OK;
}

template <int HB>
static cudaError_t md_band_launch(const double* bx, const double* by, const double* lam, const double* q,
                                  const double* cw, int Rf, int n, int M, double* scratch, double* Z, int* status,
                                  cudaStream_t s) {
  md_band_kernel<HB><<<1, 32, 0, s>>>(bx, by, lam, q, cw, Rf, n, M, scratch, Z, status);
  return cudaGetLastError();
}

// Reduced solve of dim d on the mode side, coefficients in P->d_C / P->d_c; the
// previous factor goes to P->d_Uold.
int taps_md_solve(taps_problem* P, taps_factors* U, int d) {
  int sx, sy;
  const int M = U->M;
  if (!taps_md_eligible(P, d, M, &sx, &sy) || !P->d_md) return TAPS_ERR_INVALID_ARG;
  const taps_dim* dm = P->dims[d];
  const int n = dm->nf, hb = dm->hb, Rf = P->Rf;
  const size_t MM = (size_t)M * M;
  cudaStream_t s = P->stream;
  // per-dim bases (kept across solves), their mode counts, then the solve's scratch
  double* Wm = P->d_md + (size_t)d * P->ws_M * P->ws_M;
  int* wM = (int*)(P->d_md + (size_t)TAPS_MAX_DIMS * P->ws_M * P->ws_M) + d;
  double* lam = P->d_md + (size_t)TAPS_MAX_DIMS * P->ws_M * P->ws_M + TAPS_MAX_DIMS;
  double* cw = lam + M;
  double* Z = cw + (size_t)Rf * M;
  double* scratch = Z + (size_t)P->nf_max * M;
  const size_t bsz = (size_t)n * dm->nb;
  const double* bx = dm->d_band + (size_t)P->ops[d][sx] * bsz;
  const double* by = sy >= 0 ? dm->d_band + (size_t)P->ops[d][sy] * bsz : bx;   // lam = 0 without Y
  int tk = prof_begin(P, TAPS_PROF_MODEDIAG);
  md_eig_kernel<<<1, MD_THREADS, 0, s>>>(P->d_C + (size_t)sx * MM, sy >= 0 ? P->d_C + (size_t)sy * MM : nullptr,
                                          P->d_c, Rf, M, Wm, wM, lam, cw, P->d_status);
  cudaError_t ce = cudaSuccess;
  switch (hb) {
    case 1: ce = md_band_launch<1>(bx, by, lam, P->d_q[d], cw, Rf, n, M, scratch, Z, P->d_status, s); break;
    case 2: ce = md_band_launch<2>(bx, by, lam, P->d_q[d], cw, Rf, n, M, scratch, Z, P->d_status, s); break;
    case 3: ce = md_band_launch<3>(bx, by, lam, P->d_q[d], cw, Rf, n, M, scratch, Z, P->d_status, s); break;
    case 4: ce = md_band_launch<4>(bx, by, lam, P->d_q[d], cw, Rf, n, M, scratch, Z, P->d_status, s); break;
    default: ce = md_band_launch<5>(bx, by, lam, P->d_q[d], cw, Rf, n, M, scratch, Z, P->d_status, s); break;
  }
  TAPS_CUDA(ce);
  const long long nM = (long long)n * M;
  md_out_kernel<<<(unsigned)((nM + 255) / 256), 256, 0, s>>>(Z, Wm, n, M, U->d_U[d], P->d_Uold);
  P->prof->launches[TAPS_PROF_MODEDIAG] += 2;
  // algorithmic flops: ~10 M^3 for the generalised eigenproblem, the eliminations and
  // substitutions (2 HB^2 + 6 HB per row and system), the right-hand sides and the
  // output transform
  const double Md = M;
  prof_end(P, TAPS_PROF_MODEDIAG, tk,
           10.0 * Md * Md * Md + Md * n * (2.0 * hb * hb + 6.0 * hb + 2.0 * Rf) + 2.0 * (double)nM * M,
           8.0 * (2.0 * bsz + (double)Rf * n + 3.0 * (double)nM + (double)n * (hb + 1) * M));
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}
