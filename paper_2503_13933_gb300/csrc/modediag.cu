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
//   md_prep_kernel   every system's band rows Op_X + lam_j Op_Y and right-hand side,
//                    in parallel over rows, band entries and systems.
//   md_band_kernel   thread j: Gaussian elimination without pivoting of the banded
//                    system (half-bandwidth HB) with the active rows in a register
//                    ring, then back substitution; Z is n_d x M row-major.
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
  // (its rotation is the identity; the padding row and column of S are zero)
  const int N = M + (M & 1), half = N / 2;
  if (N > M) {
    for (int j = tid; j < N; j += nt) {
      S[M][j] = 0.0;
      S[j][M] = 0.0;
    }
    __syncthreads();
  }
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
      // S <- J^T S J by 2 x 2 blocks of the round's pairs (k <= l; the lower block is
      // the transpose, the annihilated entry of a diagonal block is set to zero), and
      // V <- V J by row pairs, in one pass: the blocks and the row pairs are disjoint
      for (int idx = tid; idx < half * half; idx += nt) {
        const int k = idx / half, l = idx % half;
        if (k > l) continue;
        const double sk = rs[k], sl = rs[l];
        if (sk == 0.0 && sl == 0.0) continue;
        const double ck = rc[k], cl = rc[l];
        const int pk = rp[k], qk = rq[k], pl = rp[l], ql = rq[l];
        // B J_l
        const double b00 = S[pk][pl], b01 = S[pk][ql], b10 = S[qk][pl], b11 = S[qk][ql];
        const double t00 = cl * b00 - sl * b01, t01 = sl * b00 + cl * b01;
        const double t10 = cl * b10 - sl * b11, t11 = sl * b10 + cl * b11;
        // J_k^T (B J_l)
        const double n00 = ck * t00 - sk * t10, n01 = ck * t01 - sk * t11;
        const double n10 = sk * t00 + ck * t10, n11 = sk * t01 + ck * t11;
        if (k == l) {
          S[pk][pk] = n00;
          S[qk][qk] = n11;
          S[pk][qk] = 0.0;
          S[qk][pk] = 0.0;
        } else {
          S[pk][pl] = n00;
          S[pk][ql] = n01;
          S[qk][pl] = n10;
          S[qk][ql] = n11;
          S[pl][pk] = n00;
          S[ql][pk] = n01;
          S[pl][qk] = n10;
          S[ql][qk] = n11;
        }
      }
      for (int idx = tid; idx < half * M; idx += nt) {
        const int l = idx / M, i = idx % M;
        const double sl = rs[l];
        if (sl != 0.0) {
          const double cl = rc[l];
          const int pl = rp[l], ql = rq[l];
          const double vp = V[i][pl], vq = V[i][ql];
          V[i][pl] = cl * vp - sl * vq;
          V[i][ql] = sl * vp + cl * vq;
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

// The same generalised eigenproblem for M in (32, TAPS_MAX_M]: the M x M matrices no
// longer fit in shared memory together, so only S (the matrix the Jacobi rounds rotate,
// Np x (Np + 1) with Np = M rounded up to even) stays in shared memory; L, the rotated
// basis V (column-major, so that a round's row-pair updates are coalesced), T and the
// previous basis P live in a global workspace gw of 4 M^2 doubles (L2-resident).  The
// steps and their arithmetic are those of md_eig_kernel; W^T c_r is left to
// md_cw_kernel, spread over many CTAs.
#define MDB_THREADS 512
#define MDC_THREADS 1024   // md_core_kernel: more threads shorten each one's chain of pair updates per round
#define MDB_SMEM_SV_MAX (220 * 1024)   // S and V together in dynamic shared memory up to this size
// VSH: the basis V also lives in shared memory, after S (when both fit: Np <= 116);
// its round-by-round row-pair updates are then shared-memory traffic instead of L2
// round trips, which bound the global variant.
template <bool VSH>
__global__ void __launch_bounds__(MDB_THREADS) md_eig_big_kernel(const double* __restrict__ CX,
                                                                 const double* __restrict__ CY, int M,
                                                                 double* __restrict__ Wio, int* __restrict__ wM,
                                                                 double* __restrict__ lam, double* __restrict__ gw,
                                                                 int* status) {
  extern __shared__ __align__(16) double Ssh[];
  __shared__ double linv[TAPS_MAX_M];
  __shared__ double rc[TAPS_MAX_M / 2], rs[TAPS_MAX_M / 2];
  __shared__ int rp[TAPS_MAX_M / 2], rq[TAPS_MAX_M / 2];
  __shared__ float rcf[TAPS_MAX_M / 2], rsf[TAPS_MAX_M / 2];
  __shared__ int rotated, failed;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int Np = M + (M & 1), ld = Np + 1;
  const size_t MM = (size_t)M * M;
  double* L = gw;            // row-major [M][M], lower triangle used
  double* Vt = VSH ? Ssh + (size_t)Np * ld : gw + MM;   // column-major basis: Vt[c * M + r] = V[r][c]
  double* T = gw + 2 * MM;   // row-major temporary
  double* Pw = gw + 3 * MM;  // row-major previous basis (identity when cold)
#define SB(i, j) Ssh[(size_t)(i) * ld + (j)]
  const bool warm0 = (*wM == M);
  if (tid == 0) failed = 0;
  // With V in shared memory a first pass of FP32 rotations (the FP64 pipe of one SM
  // bounds FP64 rounds: ~4 flop per cycle) finds the basis P <- P L^-T V_32 of the
  // (previous-basis-transformed, when warm) pencil; the FP64 pass then starts from that
  // basis, and its rotations finish in two or three sweeps.  The result is the FP64
  // pass's, to FP64 accuracy.
  const int npass = VSH ? 2 : 1;
  for (int pass = 0; pass < npass; ++pass) {
  const bool warm = warm0 || pass == 1;
  const bool f32 = npass == 2 && pass == 0;
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    L[idx] = 0.5 * (CX[i * M + j] + CX[j * M + i]);
    SB(i, j) = CY ? 0.5 * (CY[i * M + j] + CY[j * M + i]) : 0.0;
    if (pass == 0) Pw[idx] = warm ? Wio[idx] : (i == j ? 1.0 : 0.0);
  }
  __syncthreads();
  if (warm) {   // L <- P^T C_X P, S <- P^T C_Y P (through T)
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += L[i * M + k] * Pw[k * M + j];
      T[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += Pw[k * M + i] * T[k * M + j];
      L[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += SB(i, k) * Pw[k * M + j];
      T[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += Pw[k * M + i] * T[k * M + j];
      SB(i, j) = s;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      if (i < j) {
        const double a = 0.5 * (L[i * M + j] + L[j * M + i]), b = 0.5 * (SB(i, j) + SB(j, i));
        L[i * M + j] = a;
        L[j * M + i] = a;
        SB(i, j) = b;
        SB(j, i) = b;
      }
    }
    __syncthreads();
  }
  // Cholesky with the same pivot floor as md_eig_kernel
  double dmax = 0.0;
  for (int k = 0; k < M; ++k) dmax = fmax(dmax, fabs(L[k * M + k]));
  const double floor_piv = 64.0 * 1.1102230246251565e-16 * dmax;
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      double piv = L[k * M + k];
      if (!isfinite(piv) || !(dmax > 0.0) || !isfinite(dmax) || piv < -1e-8 * dmax) {
        taps_flag(status, TAPS_DEV_SINGULAR);
        failed = 1;
        piv = 1.0;
      } else if (piv < floor_piv) {
        piv = floor_piv;
      }
      const double r = sqrt(piv);
      L[k * M + k] = r;
      linv[k] = taps_rcp(r);
    }
    __syncthreads();
    const double il = linv[k];
    for (int i = k + 1 + tid; i < M; i += nt) L[i * M + k] *= il;
    __syncthreads();
    const int w = M - k - 1;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int i = k + 1 + idx / w, j = k + 1 + idx % w;
      if (j <= i) L[i * M + j] -= L[i * M + k] * L[j * M + k];
    }
    __syncthreads();
  }
  // X = L^-1 C_Y into T (thread per column), then S = L^-1 X^T (thread per column)
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = SB(i, col);
      for (int j = 0; j < i; ++j) s -= L[i * M + j] * T[j * M + col];
      T[i * M + col] = s * linv[i];
    }
  }
  __syncthreads();
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = T[col * M + i];
      for (int j = 0; j < i; ++j) s -= L[i * M + j] * SB(j, col);
      SB(i, col) = s * linv[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    if (i < j) {
      const double a = 0.5 * (SB(i, j) + SB(j, i));
      SB(i, j) = a;
      SB(j, i) = a;
    }
    Vt[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  const int N = Np, half = N / 2;
  if (f32) {
    // S in FP32 in V's region, the FP32 basis (column-major) in S's region
    float* S32 = reinterpret_cast<float*>(Vt);
    float* V32 = reinterpret_cast<float*>(Ssh);
    for (int idx = tid; idx < Np * ld; idx += nt) {
      const int i = idx / ld, j = idx - i * ld;
      S32[idx] = (i < M && j < M) ? (float)SB(i, j) : 0.f;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) V32[idx] = (idx / M == idx % M) ? 1.f : 0.f;
    __syncthreads();
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
          float cs = 1.f, sn = 0.f;
          if (q < M) {
            const float apq = S32[p * ld + q], app = S32[p * ld + p], aqq = S32[q * ld + q];
            if (fabsf(apq) > 6.0e-8f * sqrtf(fabsf(app * aqq)) && fabsf(apq) > 1e-30f) {
              const float th = (aqq - app) / (2.f * apq);
              float t;
              if (fabsf(th) > 1e18f) {
                t = 0.5f / th;
              } else {
                t = 1.f / (fabsf(th) + sqrtf(th * th + 1.f));
                if (th < 0.f) t = -t;
              }
              cs = 1.f / sqrtf(t * t + 1.f);
              sn = t * cs;
              rotated = 1;
            }
          }
          rcf[tid] = cs;
          rsf[tid] = sn;
          rp[tid] = p;
          rq[tid] = q;
        }
        __syncthreads();
        for (int idx = tid; idx < half * half; idx += nt) {
          const int k = idx / half, l = idx % half;
          if (k > l) continue;
          const float sk = rsf[k], sl = rsf[l];
          if (sk == 0.f && sl == 0.f) continue;
          const float ck = rcf[k], cl = rcf[l];
          const int pk = rp[k], qk = rq[k], pl = rp[l], ql = rq[l];
          const float b00 = S32[pk * ld + pl], b01 = S32[pk * ld + ql], b10 = S32[qk * ld + pl],
                      b11 = S32[qk * ld + ql];
          const float t00 = cl * b00 - sl * b01, t01 = sl * b00 + cl * b01;
          const float t10 = cl * b10 - sl * b11, t11 = sl * b10 + cl * b11;
          const float n00 = ck * t00 - sk * t10, n01 = ck * t01 - sk * t11;
          const float n10 = sk * t00 + ck * t10, n11 = sk * t01 + ck * t11;
          if (k == l) {
            S32[pk * ld + pk] = n00;
            S32[qk * ld + qk] = n11;
            S32[pk * ld + qk] = 0.f;
            S32[qk * ld + pk] = 0.f;
          } else {
            S32[pk * ld + pl] = n00;
            S32[pk * ld + ql] = n01;
            S32[qk * ld + pl] = n10;
            S32[qk * ld + ql] = n11;
            S32[pl * ld + pk] = n00;
            S32[ql * ld + pk] = n01;
            S32[pl * ld + qk] = n10;
            S32[ql * ld + qk] = n11;
          }
        }
        for (int idx = tid; idx < half * M; idx += nt) {
          const int l = idx / M, i = idx % M;
          const float sl = rsf[l];
          if (sl != 0.f) {
            const float cl = rcf[l];
            const int pl = rp[l], ql = rq[l];
            if (ql < M) {
              const float vp = V32[pl * M + i], vq = V32[ql * M + i];
              V32[pl * M + i] = cl * vp - sl * vq;
              V32[ql * M + i] = sl * vp + cl * vq;
            }
          }
        }
        __syncthreads();
      }
      if (!rotated) break;
      __syncthreads();
    }
    // X = L^-T V_32 (FP64; thread per column, bottom row first) into T, then
    // P <- P X (through L, free until the FP64 pass reloads it): the FP64 pass's start
    if (tid < M) {
      const int col = tid;
      for (int i = M - 1; i >= 0; --i) {
        double s = (double)V32[col * M + i];
        for (int j = i + 1; j < M; ++j) s -= L[j * M + i] * T[j * M + col];
        T[i * M + col] = s * linv[i];
      }
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) {
      const int i = idx / M, j = idx % M;
      double s = 0.0;
      for (int k = 0; k < M; ++k) s += Pw[i * M + k] * T[k * M + j];
      L[idx] = s;
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) Pw[idx] = L[idx];
    __syncthreads();
    continue;
  }
  if (N > M) {
    for (int j = tid; j < N; j += nt) {
      SB(M, j) = 0.0;
      SB(j, M) = 0.0;
    }
    __syncthreads();
  }
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
          const double apq = SB(p, q), app = SB(p, p), aqq = SB(q, q);
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
      for (int idx = tid; idx < half * half; idx += nt) {
        const int k = idx / half, l = idx % half;
        if (k > l) continue;
        const double sk = rs[k], sl = rs[l];
        if (sk == 0.0 && sl == 0.0) continue;
        const double ck = rc[k], cl = rc[l];
        const int pk = rp[k], qk = rq[k], pl = rp[l], ql = rq[l];
        const double b00 = SB(pk, pl), b01 = SB(pk, ql), b10 = SB(qk, pl), b11 = SB(qk, ql);
        const double t00 = cl * b00 - sl * b01, t01 = sl * b00 + cl * b01;
        const double t10 = cl * b10 - sl * b11, t11 = sl * b10 + cl * b11;
        const double n00 = ck * t00 - sk * t10, n01 = ck * t01 - sk * t11;
        const double n10 = sk * t00 + ck * t10, n11 = sk * t01 + ck * t11;
        if (k == l) {
          SB(pk, pk) = n00;
          SB(qk, qk) = n11;
          SB(pk, qk) = 0.0;
          SB(qk, pk) = 0.0;
        } else {
          SB(pk, pl) = n00;
          SB(pk, ql) = n01;
          SB(qk, pl) = n10;
          SB(qk, ql) = n11;
          SB(pl, pk) = n00;
          SB(ql, pk) = n01;
          SB(pl, qk) = n10;
          SB(ql, qk) = n11;
        }
      }
      // V <- V J: columns p_l, q_l of V are rows p_l, q_l of Vt (coalesced over i)
      for (int idx = tid; idx < half * M; idx += nt) {
        const int l = idx / M, i = idx % M;
        const double sl = rs[l];
        if (sl != 0.0) {
          const double cl = rc[l];
          const int pl = rp[l], ql = rq[l];
          if (ql < M) {
            const double vp = Vt[(size_t)pl * M + i], vq = Vt[(size_t)ql * M + i];
            Vt[(size_t)pl * M + i] = cl * vp - sl * vq;
            Vt[(size_t)ql * M + i] = sl * vp + cl * vq;
          }
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
    double* v = Vt + (size_t)col * M;
    for (int i = M - 1; i >= 0; --i) {
      double s = v[i];
      for (int j = i + 1; j < M; ++j) s -= L[j * M + i] * v[j];
      v[i] = s * linv[i];
    }
  }
  __syncthreads();
  // W = P W_inner
  bool finite = true;
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    double s = 0.0;
    for (int k = 0; k < M; ++k) s += Pw[i * M + k] * Vt[(size_t)j * M + k];
    finite &= isfinite(s);
    T[idx] = s;
  }
  __syncthreads();
  for (int idx = tid; idx < M * M; idx += nt) Wio[idx] = T[idx];
  if (!finite) failed = 1;
  for (int j = tid; j < M; j += nt) lam[j] = SB(j, j);
  __syncthreads();
  if (tid == 0) *wM = failed ? 0 : M;
  }   // pass
#undef SB
}

// The mode-side eigen-solve split across launches (32 < M, S and V together in shared
// memory): the pencil transforms and basis products are FP64 GEMMs on many CTAs
// (md_gemm_kernel), and one CTA per pass does only what is sequential -- the Cholesky
// factorisation, S = L^-1 C_Y L^-T and the rotations.  md_core_kernel takes the
// (transformed) pencil (C_X, C_Y) and writes X = L^-T V: with F32 the rotations run in
// FP32 (the FP64 pipe of one SM bounds FP64 rounds) and X only seeds the FP64 pass;
// without, they run in FP64 to convergence and X, diag(S) are the pass's basis and
// eigenvalues.
template <bool F32>
__global__ void __launch_bounds__(MDC_THREADS) md_core_kernel(const double* __restrict__ CX,
                                                              const double* __restrict__ CY, int M,
                                                              double* __restrict__ Xout, int* __restrict__ wM,
                                                              double* __restrict__ lam, double* __restrict__ gw,
                                                              int* status, const int* __restrict__ skip,
                                                              int* __restrict__ floored_out) {
  extern __shared__ __align__(16) double Ssh[];
  __shared__ double linv[TAPS_MAX_M];
  __shared__ double rc[TAPS_MAX_M / 2], rs[TAPS_MAX_M / 2];
  __shared__ int rp[TAPS_MAX_M / 2], rq[TAPS_MAX_M / 2];
  __shared__ float rcf[TAPS_MAX_M / 2], rsf[TAPS_MAX_M / 2];
  __shared__ int rotated, failed, floored;
  __shared__ float smax32;
  __shared__ double rmin_s, rmax_s;
  if (skip && *skip) return;   // the refinement already delivered the basis
  const int tid = threadIdx.x, nt = blockDim.x;
  const int Np = M + (M & 1), ld = Np + 1;
  const size_t MM = (size_t)M * M;
  double* L = gw;                        // row-major [M][M], lower triangle used
  double* Vt = Ssh + (size_t)Np * ld;    // column-major basis: Vt[c * M + r] = V[r][c]
  double* T = gw + 2 * MM;               // row-major temporary
#define SB(i, j) Ssh[(size_t)(i) * ld + (j)]
  if (tid == 0) {
    failed = floored = 0;
    rmin_s = INFINITY;
    rmax_s = 0.0;
  }
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    L[idx] = 0.5 * (CX[i * M + j] + CX[j * M + i]);
    SB(i, j) = CY ? 0.5 * (CY[i * M + j] + CY[j * M + i]) : 0.0;
  }
  __syncthreads();
  // Cholesky with the same pivot floor as md_eig_kernel
  double dmax = 0.0;
  for (int k = 0; k < M; ++k) dmax = fmax(dmax, fabs(L[k * M + k]));
  const double floor_piv = 64.0 * 1.1102230246251565e-16 * dmax;
  for (int k = 0; k < M; ++k) {
    if (tid == 0) {
      double piv = L[k * M + k];
      if (!isfinite(piv) || !(dmax > 0.0) || !isfinite(dmax) || piv < -1e-8 * dmax) {
        taps_flag(status, TAPS_DEV_SINGULAR);
        failed = 1;
        piv = 1.0;
      } else if (piv < floor_piv) {
        piv = floor_piv;
        floored = 1;
      }
      const double r = sqrt(piv);
      L[k * M + k] = r;
      linv[k] = taps_rcp(r);
      rmin_s = fmin(rmin_s, r);
      rmax_s = fmax(rmax_s, r);
    }
    __syncthreads();
    const double il = linv[k];
    for (int i = k + 1 + tid; i < M; i += nt) L[i * M + k] *= il;
    __syncthreads();
    const int w = M - k - 1;
    for (int idx = tid; idx < w * w; idx += nt) {
      const int i = k + 1 + idx / w, j = k + 1 + idx % w;
      if (j <= i) L[i * M + j] -= L[i * M + k] * L[j * M + k];
    }
    __syncthreads();
  }
  const int N = Np, half = N / 2;
  if (F32) {
    // The seed is formed in FP32 throughout (FP32 dependent latency is a small fraction of
    // FP64's): L and T = L^-1 C_Y in V's region, S = L^-1 T^T then in S's region (C_Y,
    // read once, is dead by then), the basis V_32 (column-major) in V's region.  Its
    // error, ~kappa(L) 2^-24 against the spectral gaps, is what the FP64 corrections
    // remove.
    float* L32 = reinterpret_cast<float*>(Vt);   // [M][M]
    float* T32 = L32 + (size_t)M * M;             // [M][M]
    float* S32 = reinterpret_cast<float*>(Ssh);   // [Np][ld]
    float* V32 = reinterpret_cast<float*>(Vt);    // [M][M], after L32 and T32
    // FP32 transforms only while L is well conditioned (its diagonal within a factor 64):
    // their error grows with kappa(L); otherwise the FP64 transforms, then S to FP32
    const bool tr32 = rmax_s <= 64.0 * rmin_s;
    if (tr32) {
      for (int idx = tid; idx < M * M; idx += nt) {
        const int i = idx / M, j = idx - i * M;
        L32[idx] = (j <= i) ? (float)L[idx] : 0.f;
      }
      __syncthreads();
      if (tid < M) {   // T = L^-1 C_Y, thread per column
        const int col = tid;
        for (int i = 0; i < M; ++i) {
          float a = (float)SB(i, col);
          for (int j = 0; j < i; ++j) a = fmaf(-L32[i * M + j], T32[j * M + col], a);
          T32[i * M + col] = a * (float)linv[i];
        }
      }
      __syncthreads();
      if (tid < M) {   // S = L^-1 T^T, thread per column, into S's region as FP32
        const int col = tid;
        for (int i = 0; i < M; ++i) {
          float a = T32[col * M + i];
          for (int j = 0; j < i; ++j) a = fmaf(-L32[i * M + j], S32[j * ld + col], a);
          S32[i * ld + col] = a * (float)linv[i];
        }
      }
      __syncthreads();
    } else {
      // X = L^-1 C_Y into T (thread per column), then S = L^-1 X^T (thread per column)
      if (tid < M) {
        const int col = tid;
        for (int i = 0; i < M; ++i) {
          double s = SB(i, col);
          for (int j = 0; j < i; ++j) s -= L[i * M + j] * T[j * M + col];
          T[i * M + col] = s * linv[i];
        }
      }
      __syncthreads();
      if (tid < M) {
        const int col = tid;
        for (int i = 0; i < M; ++i) {
          double s = T[col * M + i];
          for (int j = 0; j < i; ++j) s -= L[i * M + j] * SB(j, col);
          SB(i, col) = s * linv[i];
        }
      }
      __syncthreads();
      // S (FP64) to FP32 in place: every thread reads its entries before any is written
      // (16 per thread cover Np (Np + 1) <= 116 x 117 entries with the 1024 threads)
      float sv[16];
      const int per = (Np * ld + nt - 1) / nt;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + u * nt;
        sv[u] = (u < per && idx < Np * ld) ? (float)Ssh[idx] : 0.f;
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        const int idx = tid + u * nt;
        if (u < per && idx < Np * ld) S32[idx] = sv[u];
      }
      __syncthreads();
    }
    for (int idx = tid; idx < Np * ld; idx += nt) {   // symmetric part; zero padding
      const int i = idx / ld, j = idx - i * ld;
      if (i >= M || j >= M) S32[idx] = 0.f;
      else if (i < j) {
        const float a = 0.5f * (S32[idx] + S32[j * ld + i]);
        S32[idx] = a;
        S32[j * ld + i] = a;
      }
    }
    __syncthreads();
    for (int idx = tid; idx < M * M; idx += nt) V32[idx] = (idx / M == idx % M) ? 1.f : 0.f;
    if (tid < 32) {   // the largest diagonal magnitude: the absolute floor of the rotations
      float m = 0.f;
      for (int i = tid; i < M; i += 32) m = fmaxf(m, fabsf(S32[i * ld + i]));
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (tid == 0) smax32 = m;
    }
    __syncthreads();
    // The FP32 basis only seeds the FP64 corrections, which converge from an error of
    // ~1e-3 against the spectral gaps: a pair is rotated while its coupling exceeds
    // 1e-5 of its diagonal entries (and 1e-7 of the largest one).  A tighter threshold
    // would chase FP32 rounding noise (~6e-8 of a row's scale) and keep rotating.
    const float abs_floor = 1e-7f * smax32;
    const int lane = tid & 31, wid = tid >> 5, nw = nt >> 5;
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
          float cs = 1.f, sn = 0.f;
          if (q < M) {
            const float apq = S32[p * ld + q], app = S32[p * ld + p], aqq = S32[q * ld + q];
            if (fabsf(apq) > 1e-5f * sqrtf(fabsf(app * aqq)) && fabsf(apq) > abs_floor && fabsf(apq) > 1e-30f) {
              // the rotation's chain is the round's serial part: approximate quotient,
              // square root and reciprocal square root (cs^2 + sn^2 = 1 to FP32 accuracy)
              const float th = __fdividef(aqq - app, 2.f * apq);
              float t;
              if (fabsf(th) > 1e18f) {
                t = __fdividef(0.5f, th);
              } else {
                t = __fdividef(1.f, fabsf(th) + __fsqrt_rn(fmaf(th, th, 1.f)));
                if (th < 0.f) t = -t;
              }
              cs = rsqrtf(fmaf(t, t, 1.f));
              sn = t * cs;
              rotated = 1;
            }
          }
          rcf[tid] = cs;
          rsf[tid] = sn;
          rp[tid] = p;
          rq[tid] = q;
        }
        __syncthreads();
        // the round's rotations applied as two passes over contiguous data (rows, then
        // columns: S <- J^T S J), so that shared-memory accesses do not collide in
        // banks (row stride ld is odd), with the basis rows of V^T in the row pass.
        // Warp w takes the pairs w, w + 32, ... (its rotation read once), lanes the
        // entries of the pair's rows or columns.
        for (int l = wid; l < half; l += nw) {
          const float sl = rsf[l];
          if (sl == 0.f) continue;
          const float cl = rcf[l];
          const int pl = rp[l], ql = rq[l];
          float* Sp = S32 + pl * ld;
          float* Sq = S32 + ql * ld;
#pragma unroll 4
          for (int c = lane; c < N; c += 32) {
            const float a = Sp[c], bq = Sq[c];
            Sp[c] = cl * a - sl * bq;
            Sq[c] = sl * a + cl * bq;
          }
          if (ql < M) {
            float* Vp = V32 + pl * M;
            float* Vq = V32 + ql * M;
#pragma unroll 4
            for (int c = lane; c < M; c += 32) {
              const float vp = Vp[c], vq = Vq[c];
              Vp[c] = cl * vp - sl * vq;
              Vq[c] = sl * vp + cl * vq;
            }
          }
        }
        __syncthreads();
        for (int l = wid; l < half; l += nw) {
          const float sl = rsf[l];
          if (sl == 0.f) continue;
          const float cl = rcf[l];
          const int pl = rp[l], ql = rq[l];
#pragma unroll 4
          for (int r2 = lane; r2 < N; r2 += 32) {
            const float a = S32[r2 * ld + pl], bq = S32[r2 * ld + ql];
            S32[r2 * ld + pl] = (r2 == ql) ? 0.f : cl * a - sl * bq;
            S32[r2 * ld + ql] = (r2 == pl) ? 0.f : sl * a + cl * bq;
          }
        }
        __syncthreads();
      }
      if (!rotated) break;
      __syncthreads();
    }
    if (tr32) {
      // X = L^-T V_32 (thread per column, bottom row first), in FP32 with L reloaded into
      // S's region (dead now) and X beside it
      float* Lb = S32;
      float* X32 = S32 + (size_t)M * M;
      for (int idx = tid; idx < M * M; idx += nt) {
        const int i = idx / M, j = idx - i * M;
        Lb[idx] = (j <= i) ? (float)L[idx] : 0.f;
      }
      __syncthreads();
      if (tid < M) {
        const int col = tid;
        for (int i = M - 1; i >= 0; --i) {
          float a = V32[col * M + i];
          for (int j = i + 1; j < M; ++j) a = fmaf(-Lb[j * M + i], X32[j * M + col], a);
          X32[i * M + col] = a * (float)linv[i];
        }
      }
      __syncthreads();
      for (int idx = tid; idx < M * M; idx += nt) Xout[idx] = (double)X32[idx];
    } else {   // X = L^-T V_32 in FP64 (thread per column, bottom row first)
      if (tid < M) {
        const int col = tid;
        for (int i = M - 1; i >= 0; --i) {
          double a = (double)V32[col * M + i];
          for (int j = i + 1; j < M; ++j) a -= L[j * M + i] * Xout[j * M + col];
          Xout[i * M + col] = a * linv[i];
        }
      }
    }
    if (tid == 0 && floored_out) *floored_out = floored | failed;
    return;
  }
  // X = L^-1 C_Y into T (thread per column), then S = L^-1 X^T (thread per column)
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = SB(i, col);
      for (int j = 0; j < i; ++j) s -= L[i * M + j] * T[j * M + col];
      T[i * M + col] = s * linv[i];
    }
  }
  __syncthreads();
  if (tid < M) {
    const int col = tid;
    for (int i = 0; i < M; ++i) {
      double s = T[col * M + i];
      for (int j = 0; j < i; ++j) s -= L[i * M + j] * SB(j, col);
      SB(i, col) = s * linv[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    if (i < j) {
      const double a = 0.5 * (SB(i, j) + SB(j, i));
      SB(i, j) = a;
      SB(j, i) = a;
    }
    Vt[idx] = (i == j) ? 1.0 : 0.0;
  }
  __syncthreads();
  if (N > M) {
    for (int j = tid; j < N; j += nt) {
      SB(M, j) = 0.0;
      SB(j, M) = 0.0;
    }
    __syncthreads();
  }
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
          const double apq = SB(p, q), app = SB(p, p), aqq = SB(q, q);
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
      for (int idx = tid; idx < half * half; idx += nt) {
        const int k = idx / half, l = idx % half;
        if (k > l) continue;
        const double sk = rs[k], sl = rs[l];
        if (sk == 0.0 && sl == 0.0) continue;
        const double ck = rc[k], cl = rc[l];
        const int pk = rp[k], qk = rq[k], pl = rp[l], ql = rq[l];
        const double b00 = SB(pk, pl), b01 = SB(pk, ql), b10 = SB(qk, pl), b11 = SB(qk, ql);
        const double t00 = cl * b00 - sl * b01, t01 = sl * b00 + cl * b01;
        const double t10 = cl * b10 - sl * b11, t11 = sl * b10 + cl * b11;
        const double n00 = ck * t00 - sk * t10, n01 = ck * t01 - sk * t11;
        const double n10 = sk * t00 + ck * t10, n11 = sk * t01 + ck * t11;
        if (k == l) {
          SB(pk, pk) = n00;
          SB(qk, qk) = n11;
          SB(pk, qk) = 0.0;
          SB(qk, pk) = 0.0;
        } else {
          SB(pk, pl) = n00;
          SB(pk, ql) = n01;
          SB(qk, pl) = n10;
          SB(qk, ql) = n11;
          SB(pl, pk) = n00;
          SB(ql, pk) = n01;
          SB(pl, qk) = n10;
          SB(ql, qk) = n11;
        }
      }
      // V <- V J: columns p_l, q_l of V are rows p_l, q_l of Vt (coalesced over i)
      for (int idx = tid; idx < half * M; idx += nt) {
        const int l = idx / M, i = idx % M;
        const double sl = rs[l];
        if (sl != 0.0) {
          const double cl = rc[l];
          const int pl = rp[l], ql = rq[l];
          if (ql < M) {
            const double vp = Vt[(size_t)pl * M + i], vq = Vt[(size_t)ql * M + i];
            Vt[(size_t)pl * M + i] = cl * vp - sl * vq;
            Vt[(size_t)ql * M + i] = sl * vp + cl * vq;
          }
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
    double* v = Vt + (size_t)col * M;
    for (int i = M - 1; i >= 0; --i) {
      double s = v[i];
      for (int j = i + 1; j < M; ++j) s -= L[j * M + i] * v[j];
      v[i] = s * linv[i];
    }
  }
  __syncthreads();
  for (int idx = tid; idx < M * M; idx += nt) {
    const int i = idx / M, j = idx % M;
    Xout[idx] = Vt[(size_t)j * M + i];
    if (!isfinite(Xout[idx])) failed = 1;
  }
  for (int j = tid; j < M; j += nt) lam[j] = SB(j, j);
  __syncthreads();
  if (tid == 0) *wM = failed ? 0 : M;
#undef SB
}

// C = op(A) B for M x M row-major FP64 matrices, a 16 x 16 output tile per CTA.  With a
// basis flag (P_mode != 0) the operand P is the dim's previous basis when it is sound
// (*wM == M) and the identity otherwise: P_mode 1: C = A P (A when cold); 2: C = P^T B
// (B when cold); 3: C = P B (B when cold).
__global__ void __launch_bounds__(256) md_gemm_kernel(const double* __restrict__ A, int transA,
                                                      const double* __restrict__ B, double* __restrict__ C, int M,
                                                      const int* __restrict__ wM, int P_mode,
                                                      const int* __restrict__ skip) {
  __shared__ double As[16][17], Bs[16][17];
  if (skip && *skip) return;   // the refinement already delivered the basis
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = blockIdx.y * 16 + ty, col = blockIdx.x * 16 + tx;
  const bool cold = P_mode != 0 && *wM != M;
  if (cold) {   // a product with the identity
    if (row < M && col < M) C[row * M + col] = (P_mode == 1) ? A[row * M + col] : B[row * M + col];
    return;
  }
  double acc = 0.0;
  for (int k0 = 0; k0 < M; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    As[ty][tx] = (row < M && ka < M) ? (transA ? A[ka * M + row] : A[row * M + ka]) : 0.0;
    Bs[ty][tx] = (kb < M && col < M) ? B[kb * M + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(As[ty][k], Bs[k][tx], acc);
    __syncthreads();
  }
  if (row < M && col < M) C[row * M + col] = acc;
}

// Refinement of an approximate eigenbasis X of the symmetric-definite pencil
// (C_Y, C_X) in FP64 by matrix products only (first-order correction, repeated):
// with R = I - X^T C_X X and S = X^T C_Y X, the exact basis is X (I + F) where, to first
// order, F + F^T = R (C_X-orthonormality) and S + F^T D + D F is diagonal (D = diag of
// the Rayleigh quotients lam_i = S_ii / (1 - R_ii)), i.e. F_ii = R_ii / 2 and
// F_ij = (S_ij + lam_j R_ij) / (lam_j - lam_i) for i != j.  Each correction is about
// the square of the previous one while the error is small against the gaps of lam
// (the FP32 seed's error is ~kappa(L) 2^-24 against them; three or four corrections
// reach the FP64 rounding floor, at most five are taken).  A step whose largest |F| exceeds MR_FAIL (no quadratic regime: a cluster
// or a poor start) ends the refinement unaccepted, and so does a non-finite entry;
// once max |F| <= MR_DONE the corrected basis goes to Wout, lam to lam_out and *acc
// = 1 (the FP64 rotation pass is then skipped).  Not attempted when the FP32 pass
// raised a Cholesky pivot of C_X to its floor (the rotation pass's regularised
// pencil, not the exact one, is then the solve's).  One cooperative launch; phases
// are separated by bounded grid barriers, and every CTA takes the same decisions from
// the same global maximum.
#define MR_THREADS 256
#define MR_MAX_STEPS 5
#define MR_FAIL 0.1
#define MR_DONE 1e-9
struct MrBufs {
  double *Xa, *Xb, *T1, *T2, *A, *B, *F;
  unsigned long long* maxbits;   // [MR_MAX_STEPS] bit patterns of non-negative doubles
  unsigned* bar;                 // grid barrier (zeroed before the launch)
};

// C[tile] = op(P) Q for one 16 x 16 output tile; sym: P is the symmetric part of a
// coefficient matrix (0.5 (P + P^T)); transP: P^T.  Accumulation over k in order.
__device__ __forceinline__ void mr_tile(const double* __restrict__ Pm, int sym, int transP,
                                        const double* __restrict__ Q, double* __restrict__ C, int M, int ti,
                                        int tj, double (*Ps)[17], double (*Qs)[17], const double* __restrict__ Add) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int row = ti * 16 + ty, col = tj * 16 + tx;
  double acc = 0.0;
  for (int k0 = 0; k0 < M; k0 += 16) {
    const int ka = k0 + tx, kb = k0 + ty;
    double pv = 0.0;
    if (row < M && ka < M) {
      if (sym) pv = 0.5 * (Pm[row * M + ka] + Pm[ka * M + row]);
      else pv = transP ? Pm[ka * M + row] : Pm[row * M + ka];
    }
    Ps[ty][tx] = pv;
    Qs[ty][tx] = (kb < M && col < M) ? Q[kb * M + col] : 0.0;
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 16; ++k) acc = fma(Ps[ty][k], Qs[k][tx], acc);
    __syncthreads();
  }
  if (row < M && col < M) C[row * M + col] = Add ? Add[row * M + col] + acc : acc;
}

__device__ __forceinline__ double mr_max_read(const unsigned long long* p) {
  return __longlong_as_double((long long)*(volatile const unsigned long long*)p);
}

__global__ void __launch_bounds__(MR_THREADS) md_refine_kernel(const double* __restrict__ CX,
                                                              const double* __restrict__ CY, int M,
                                                              const double* __restrict__ X0, MrBufs b,
                                                              double* __restrict__ Wout, double* __restrict__ lam_out,
                                                              int* wM, int* acc, const int* __restrict__ floored,
                                                              int* status) {
  __shared__ double Ps[16][17], Qs[16][17];
  __shared__ double red[MR_THREADS / 32];
  const int nt = (M + 15) / 16, ntt = nt * nt;
  const unsigned nb = gridDim.x;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *acc = 0;
    for (int k = 0; k < MR_MAX_STEPS; ++k) b.maxbits[k] = 0ull;
  }
  // a Cholesky pivot of the FP32 pass raised to the floor: C_X is numerically
  // singular on the modes, and the FP64 rotation pass (with the same floor) decides
  if (*floored) return;
  const double* X = X0;
  for (int step = 0; step < MR_MAX_STEPS; ++step) {
    double* Xn = (step & 1) ? b.Xb : b.Xa;
    // T1 = sym(C_X) X, T2 = sym(C_Y) X (C_Y absent: T2 unused)
    for (int it = blockIdx.x; it < 2 * ntt; it += nb) {
      const int mat = it / ntt, t = it % ntt;
      if (mat == 1 && !CY) continue;
      mr_tile(mat ? CY : CX, 1, 0, X, mat ? b.T2 : b.T1, M, t / nt, t % nt, Ps, Qs, nullptr);
    }
    grid_barrier(b.bar, status, nb);
    // A = X^T T1, B = X^T T2
    for (int it = blockIdx.x; it < 2 * ntt; it += nb) {
      const int mat = it / ntt, t = it % ntt;
      if (mat == 1 && !CY) continue;
      mr_tile(X, 0, 1, mat ? b.T2 : b.T1, mat ? b.B : b.A, M, t / nt, t % nt, Ps, Qs, nullptr);
    }
    grid_barrier(b.bar, status, nb);
    // F and its largest magnitude (non-finite entries count as infinite)
    double fmx = 0.0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < M * M; e += nb * blockDim.x) {
      const int i = e / M, j = e % M;
      const double Rij = (i == j ? 1.0 : 0.0) - 0.5 * (b.A[i * M + j] + b.A[j * M + i]);
      const double Rii = 1.0 - b.A[i * M + i], Rjj = 1.0 - b.A[j * M + j];
      const double Sij = CY ? 0.5 * (b.B[i * M + j] + b.B[j * M + i]) : 0.0;
      const double li = CY ? b.B[i * M + i] / (1.0 - Rii) : 0.0;
      const double lj = CY ? b.B[j * M + j] / (1.0 - Rjj) : 0.0;
      double f;
      if (i == j) {
        f = 0.5 * Rij;
        lam_out[i] = li;   // final only when this step is accepted; else the FP64 pass rewrites it
      } else {
        f = (Sij + lj * Rij) / (lj - li);
        if (!CY) f = 0.5 * Rij;
      }
      b.F[e] = f;
      const double a = fabs(f);
      fmx = isfinite(a) ? fmax(fmx, a) : INFINITY;
    }
    for (int o = 16; o > 0; o >>= 1) fmx = fmax(fmx, __shfl_xor_sync(0xffffffffu, fmx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = fmx;
    __syncthreads();
    if (threadIdx.x == 0) {
      double m = 0.0;
      for (int w = 0; w < MR_THREADS / 32; ++w) m = fmax(m, red[w]);
      atomicMax(b.maxbits + step, (unsigned long long)__double_as_longlong(m));
    }
    grid_barrier(b.bar, status, nb);
    const double mx = mr_max_read(b.maxbits + step);
    if (!(mx <= MR_FAIL)) return;   // not accepted: the FP64 rotation pass runs
    const bool done = mx <= MR_DONE;
    // X_next = X + X F (into the basis output once accepted)
    double* dst = done ? Wout : Xn;
    for (int t = blockIdx.x; t < ntt; t += nb) mr_tile(X, 0, 0, b.F, dst, M, t / nt, t % nt, Ps, Qs, X);
    if (done) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        *acc = 1;
        *wM = M;
      }
      return;
    }
    grid_barrier(b.bar, status, nb);
    X = Xn;
  }
}

// cw[r][j] = sum_m c[r][m] W[m][j] (the right-hand side's mode-side coefficients), one
// thread per entry over many CTAs.
__global__ void md_cw_kernel(const double* __restrict__ c, const double* __restrict__ Wm, int Rf, int M,
                             double* __restrict__ cw) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)Rf * M) return;
  const int r = (int)(idx / M), j = (int)(idx % M);
  const double* cr = c + (size_t)r * M;
  double s = 0.0;
  for (int m = 0; m < M; ++m) s += cr[m] * Wm[(size_t)m * M + j];
  cw[idx] = s;
}

// Padding rows below the matrix (identity rows, zero right-hand side) let the
// elimination run whole unrolled groups and read ahead without bounds tests.
#define MD_PAD 24

// Ab[(i * (2HB+2) + k) * M + j]: row i of Op_X + lam_j Op_Y in band-relative form
// (k = column - i + HB, zero outside the matrix) and, at k = 2HB+1, the right-hand side
// (F W)[i][j] = sum_r q_r[i] Wc_r[j]; rows n .. n+MD_PAD-1 are identity rows.
template <int HB>
__global__ void md_prep_kernel(const double* __restrict__ bx, const double* __restrict__ by,
                               const double* __restrict__ lam, const double* __restrict__ q,
                               const double* __restrict__ cw, int Rf, int n, int M, double* __restrict__ Ab) {
  constexpr int W2 = 2 * HB + 1, RW = W2 + 1;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long tot = (long long)(n + MD_PAD) * RW * M;
  if (idx >= tot) return;
  const int j = (int)(idx % M);
  const int k = (int)((idx / M) % RW);
  const int i = (int)(idx / ((long long)M * RW));
  double v = 0.0;
  if (i >= n) {
    v = (k == HB) ? 1.0 : 0.0;
  } else if (k < W2) {
    const int col = i + k - HB;
    if (col >= 0 && col < n) v = fma(lam[j], by[(size_t)i * W2 + k], bx[(size_t)i * W2 + k]);
  } else {
    for (int r = 0; r < Rf; ++r) v = fma(q[(size_t)r * n + i], cw[r * M + j], v);
  }
  Ab[idx] = v;
}

// Thread j < M solves (Op_X + lam_j Op_Y) z_j = (F W)_j by Gaussian elimination without
// pivoting (no fill outside the band).  The active rows i .. i+HB live in a ring of
// NS = HB+1 register rows in band-relative form, so a row keeps its storage while the
// window moves: row i+r sits in slot (i+r) mod NS, its entry in column i + c at
// HB + c - r.  The loop is unrolled by U = lcm(NS, 2) so that every slot index is a
// compile-time constant; the row entering at step i (row i+HB+1, into the pivot's slot)
// was loaded two steps earlier.  Stored per step: the pivot row scaled by the pivot's
// reciprocal, scratch[(i * (HB+1) + c) * M + j] (c = 0: right-hand side, 1..HB:
// superdiagonal); back substitution walks them upwards with the same ring.
template <int HB>
__global__ void __launch_bounds__(32) md_band_kernel(const double* __restrict__ Ab, int n, int M,
                                                     double* __restrict__ scratch, double* __restrict__ Z,
                                                     int* status) {
  constexpr int W2 = 2 * HB + 1, RW = W2 + 1, NS = HB + 1;
  constexpr int U = (NS % 2 == 0) ? NS : 2 * NS;
  const int j = blockIdx.x * 32 + threadIdx.x;   // system index (one warp per 32 systems)
  if (j >= M) return;
  const int nsteps = ((n + U - 1) / U) * U;   // <= n + U - 1; rows read <= nsteps + HB + 2
  double A[NS][W2];
  double b[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) {
    const double* row = Ab + (size_t)r * RW * M + j;
#pragma unroll
    for (int k = 0; k < W2; ++k) A[r][k] = row[(size_t)k * M];
    b[r] = row[(size_t)W2 * M];
  }
  double st[2][RW];   // staged rows: row i+HB+1 enters at step i from st[i & 1]
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const double* row = Ab + (size_t)(HB + 1 + t) * RW * M + j;
#pragma unroll
    for (int k = 0; k < RW; ++k) st[t][k] = row[(size_t)k * M];
  }
  bool bad = false;
  for (int i0 = 0; i0 < nsteps; i0 += U) {
#pragma unroll
    for (int ph = 0; ph < U; ++ph) {
      const int i = i0 + ph;
      const int P = ph % NS;
      const double piv = A[P][HB];
      const bool ok = fabs(piv) > 0.0 && isfinite(piv);
      bad |= !ok;
      const double inv = ok ? taps_rcp(piv) : 0.0;
#pragma unroll
      for (int r = 1; r <= HB; ++r) {
        const int R = (ph + r) % NS;
        const double l = A[R][HB - r] * inv;
#pragma unroll
        for (int c = 1; c <= HB; ++c) A[R][HB + c - r] -= l * A[P][HB + c];
        b[R] -= l * b[P];
      }
      double* out = scratch + (size_t)i * NS * M + j;
      out[0] = b[P] * inv;
#pragma unroll
      for (int c = 1; c <= HB; ++c) out[(size_t)c * M] = A[P][HB + c] * inv;
      // row i+HB+1 takes the pivot's slot; row i+HB+3 is staged in its place
      const int t = ph & 1;
#pragma unroll
      for (int k = 0; k < W2; ++k) A[P][k] = st[t][k];
      b[P] = st[t][W2];
      const double* row = Ab + (size_t)(i + HB + 3) * RW * M + j;
#pragma unroll
      for (int k = 0; k < RW; ++k) st[t][k] = row[(size_t)k * M];
    }
  }
  if (bad) taps_flag(status, TAPS_DEV_SINGULAR);
  // back substitution over the padded rows (their solution is zero): z_i = y_i -
  // sum_c u_ic z_{i+c}, z in a ring of NS slots, stored rows loaded two steps ahead
  double z[NS];
#pragma unroll
  for (int r = 0; r < NS; ++r) z[r] = 0.0;
  double sr[2][NS];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const double* u = scratch + (size_t)(nsteps - 1 - t) * NS * M + j;
#pragma unroll
    for (int c = 0; c < NS; ++c) sr[t][c] = u[(size_t)c * M];
  }
  for (int i0 = nsteps - U; i0 >= 0; i0 -= U) {
#pragma unroll
    for (int ph = U - 1; ph >= 0; --ph) {
      const int i = i0 + ph;
      const int t = (U - 1 - ph) & 1;   // rows nsteps-1, nsteps-2, ... alternate buffers
      // the terms of z_{i+2} .. z_{i+HB} first: only the last FMA waits for z_{i+1}
      double s = sr[t][0];
#pragma unroll
      for (int c = HB; c >= 2; --c) s -= sr[t][c] * z[(ph + c) % NS];
      s -= sr[t][1] * z[(ph + 1) % NS];
      z[ph % NS] = s;
      if (i < n) Z[(size_t)i * M + j] = s;
      const int nx = i - 2;
      if (nx >= 0) {
        const double* u = scratch + (size_t)nx * NS * M + j;
#pragma unroll
        for (int c = 0; c < NS; ++c) sr[t][c] = u[(size_t)c * M];
      }
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
  if (nops < 1 || nops > 2 || M < 1 || M > TAPS_MAX_M) return 0;
  if (P->has_weighted) return 0;   // symmetry of weighted operators is not tracked
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
  int c0, c1, nb;
  if (solver == TAPS_SOLVER_MODEDIAG) {
    if (taps_md_eligible(P, d, M, &a, &b)) return TAPS_ROUTE_MD;
    if (taps_fd_eligible(P, d, &a, &b)) return TAPS_ROUTE_FD;
    if (taps_fdw_eligible(P, d, M, &a, &b, &c0, &c1, &nb)) return TAPS_ROUTE_FDW;
    return TAPS_ROUTE_LU;
  }
  if (solver == TAPS_SOLVER_FASTDIAG) {
    if (taps_fd_eligible(P, d, &a, &b)) return TAPS_ROUTE_FD;
    if (taps_md_eligible(P, d, M, &a, &b) && P->tt.nops[d] == 2) return TAPS_ROUTE_MD;
    if (taps_fdw_eligible(P, d, M, &a, &b, &c0, &c1, &nb)) return TAPS_ROUTE_FDW;
  }
  return TAPS_ROUTE_LU;
}

// [TAPS_MAX_DIMS][M][M] bases, TAPS_MAX_DIMS ints (one double each), lam [M], W^T c
// [Rf][M], Z [nf_max][M], eliminated rows [nf_max + MD_PAD][MD_MAX_HB + 1][M], band
// rows [nf_max + MD_PAD][2 MD_MAX_HB + 2][M].  The caller zeroes it (no valid basis).
size_t taps_md_scratch_doubles(int nf_max, int M, int Rf) {
  return (size_t)TAPS_MAX_DIMS * M * M + TAPS_MAX_DIMS + M + (size_t)Rf * M + (size_t)nf_max * M +
         (size_t)(nf_max + MD_PAD) * (MD_MAX_HB + 1) * M + (size_t)(nf_max + MD_PAD) * (2 * MD_MAX_HB + 2) * M +
         (M > 32 ? (size_t)14 * M * M + 8 : 0);
}

// Forgets every dim's stored basis (the next solves start cold).  Called when a sweep
// call starts, so that the same factors always give the same rounding.
int taps_md_reset(taps_problem* P) {
  if (!P->d_md || P->ws_M < 1) return TAPS_OK;
  TAPS_CUDA(cudaMemsetAsync(P->d_md + (size_t)TAPS_MAX_DIMS * P->ws_M * P->ws_M, 0, sizeof(int) * TAPS_MAX_DIMS,
                            P->stream));
  return TAPS_OK;
}

// Shared-memory opt-in of the large-M eigen-solve (S of up to TAPS_MAX_M rows, padded);
// made with the problem's device current when its first problem is created.
int taps_md_setup(int maxsm) {
  const int need = (int)(sizeof(double) * (TAPS_MAX_M + 1) * (TAPS_MAX_M + 2));
  cudaFuncAttributes fa;
  TAPS_CUDA(cudaFuncGetAttributes(&fa, md_eig_big_kernel<false>));
  TAPS_CUDA(cudaFuncSetAttribute(md_eig_big_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::min(need, maxsm - (int)fa.sharedSizeBytes)));
  TAPS_CUDA(cudaFuncGetAttributes(&fa, md_eig_big_kernel<true>));
  TAPS_CUDA(cudaFuncSetAttribute(md_eig_big_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::min(MDB_SMEM_SV_MAX, maxsm - (int)fa.sharedSizeBytes)));
  TAPS_CUDA(cudaFuncGetAttributes(&fa, md_core_kernel<true>));
  TAPS_CUDA(cudaFuncSetAttribute(md_core_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::min(MDB_SMEM_SV_MAX, maxsm - (int)fa.sharedSizeBytes)));
  TAPS_CUDA(cudaFuncGetAttributes(&fa, md_core_kernel<false>));
  TAPS_CUDA(cudaFuncSetAttribute(md_core_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 std::min(MDB_SMEM_SV_MAX, maxsm - (int)fa.sharedSizeBytes)));
  return TAPS_OK;
}

template <int HB>
static cudaError_t md_band_launch(const double* bx, const double* by, const double* lam, const double* q,
                                  const double* cw, int Rf, int n, int M, double* Ab, double* scratch, double* Z,
                                  int* status, cudaStream_t s) {
  const long long tot = (long long)(n + MD_PAD) * (2 * HB + 2) * M;
  md_prep_kernel<HB><<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(bx, by, lam, q, cw, Rf, n, M, Ab);
  md_band_kernel<HB><<<(unsigned)((M + 31) / 32), 32, 0, s>>>(Ab, n, M, scratch, Z, status);
  return cudaGetLastError();
}

// The eigen-solve of one mode-side solve, 32 < M with S and V in shared memory: the
// pencil transforms with the previous basis (identity when *wM != M), FP32 rotations,
// the FP64 refinement, and the FP64 rotation pass when the refinement is not accepted.
// gw: 14 M^2 + 8 doubles of workspace; on return Wm, lam and *wM hold the new basis.
static int md_eig_split(const double* CX, const double* CY, int M, double* Wm, int* wM, double* lam, double* gw,
                        int* status, int num_sms, cudaStream_t s) {
  const size_t MM = (size_t)M * M;
  const int Np = M + (M & 1);
  const size_t smem_sv = sizeof(double) * ((size_t)Np * (Np + 1) + (size_t)M * M);
  double* T = gw + 2 * MM;
  double* P1 = gw + 3 * MM;
  double* CXw = gw + 4 * MM;
  double* CYw = gw + 5 * MM;
  double* X = gw + 6 * MM;
  const dim3 gg((M + 15) / 16, (M + 15) / 16);
  MrBufs rb;
  rb.Xa = gw + 7 * MM;
  rb.Xb = gw + 8 * MM;
  rb.T1 = gw + 9 * MM;
  rb.T2 = gw + 10 * MM;
  rb.A = gw + 11 * MM;
  rb.B = gw + 12 * MM;
  rb.F = gw + 13 * MM;
  rb.maxbits = (unsigned long long*)(gw + 14 * MM);
  rb.bar = (unsigned*)(gw + 14 * MM + MR_MAX_STEPS);
  int* acc = (int*)(gw + 14 * MM + MR_MAX_STEPS + 1);
  int* floored = (int*)(gw + 14 * MM + MR_MAX_STEPS + 2);
  const int* no_skip = nullptr;
  // the previous basis P (identity when cold): CXw = P^T C_X P, CYw = P^T C_Y P
  md_gemm_kernel<<<gg, 256, 0, s>>>(CX, 0, Wm, T, M, wM, 1, no_skip);
  md_gemm_kernel<<<gg, 256, 0, s>>>(Wm, 1, T, CXw, M, wM, 2, no_skip);
  if (CY) {
    md_gemm_kernel<<<gg, 256, 0, s>>>(CY, 0, Wm, T, M, wM, 1, no_skip);
    md_gemm_kernel<<<gg, 256, 0, s>>>(Wm, 1, T, CYw, M, wM, 2, no_skip);
  }
  // FP32 rotations: X, then P1 = P X
  md_core_kernel<true><<<1, MDC_THREADS, smem_sv, s>>>(CXw, CY ? CYw : nullptr, M, X, wM, lam, gw,
                                                       status, no_skip, floored);
  md_gemm_kernel<<<gg, 256, 0, s>>>(Wm, 0, X, P1, M, wM, 3, no_skip);
  // FP64 corrections of P1 by matrix products (many CTAs); accepted, they give W
  // and lam and the FP64 rotation pass below returns at once
  {
    const int ntt = ((M + 15) / 16) * ((M + 15) / 16);
    const int grid = std::max(1, std::min(2 * ntt, num_sms));
    TAPS_CUDA(cudaMemsetAsync(rb.bar, 0, 2 * sizeof(unsigned), s));
    const double* X0 = P1;
    void* args[] = {(void*)&CX, (void*)&CY, (void*)&M, (void*)&X0, (void*)&rb, (void*)&Wm,
                    (void*)&lam, (void*)&wM, (void*)&acc, (void*)&floored, (void*)&status};
    TAPS_CUDA(cudaLaunchCooperativeKernel((const void*)md_refine_kernel, dim3(grid), dim3(MR_THREADS), args, 0,
                                          s));
  }
  // FP64 rotation pass on (P1^T C_X P1, P1^T C_Y P1): X = W_inner, lam; W = P1 W_inner
  md_gemm_kernel<<<gg, 256, 0, s>>>(CX, 0, P1, T, M, wM, 0, acc);
  md_gemm_kernel<<<gg, 256, 0, s>>>(P1, 1, T, CXw, M, wM, 0, acc);
  if (CY) {
    md_gemm_kernel<<<gg, 256, 0, s>>>(CY, 0, P1, T, M, wM, 0, acc);
    md_gemm_kernel<<<gg, 256, 0, s>>>(P1, 1, T, CYw, M, wM, 0, acc);
  }
  md_core_kernel<false><<<1, MDC_THREADS, smem_sv, s>>>(CXw, CY ? CYw : nullptr, M, X, wM, lam, gw,
                                                        status, acc, nullptr);
  md_gemm_kernel<<<gg, 256, 0, s>>>(P1, 0, X, Wm, M, wM, 0, acc);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
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
  double* Ab = scratch + (size_t)(P->nf_max + MD_PAD) * (MD_MAX_HB + 1) * M;
  const size_t bsz = (size_t)n * dm->nb;
  const double* bx = dm->d_band + (size_t)P->ops[d][sx] * bsz;
  const double* by = sy >= 0 ? dm->d_band + (size_t)P->ops[d][sy] * bsz : bx;   // lam = 0 without Y
  int tk = prof_begin(P, TAPS_PROF_MODEDIAG);
  if (M <= 32) {
    md_eig_kernel<<<1, MD_THREADS, 0, s>>>(P->d_C + (size_t)sx * MM, sy >= 0 ? P->d_C + (size_t)sy * MM : nullptr,
                                            P->d_c, Rf, M, Wm, wM, lam, cw, P->d_status);
  } else {
    // the eigen-solve's workspace follows the band rows (sized for M > 32 only)
    double* gw = Ab + (size_t)(P->nf_max + MD_PAD) * (2 * MD_MAX_HB + 2) * M;
    const int Np = M + (M & 1);
    const size_t smem_s = sizeof(double) * (size_t)Np * (Np + 1);   // opted in by taps_md_setup
    const size_t smem_sv = smem_s + sizeof(double) * (size_t)M * M;
    if (smem_sv <= (size_t)MDB_SMEM_SV_MAX) {
      // transforms and basis products on many CTAs, the sequential part on one
      TAPS_TRY(md_eig_split(P->d_C + (size_t)sx * MM, sy >= 0 ? P->d_C + (size_t)sy * MM : nullptr, M, Wm, wM,
                            lam, gw, P->d_status, P->num_sms, s));
      P->prof->launches[TAPS_PROF_MODEDIAG] += sy >= 0 ? 12 : 8;
    } else {
      md_eig_big_kernel<false><<<1, MDB_THREADS, smem_s, s>>>(P->d_C + (size_t)sx * MM,
                                                              sy >= 0 ? P->d_C + (size_t)sy * MM : nullptr, M, Wm,
                                                              wM, lam, gw, P->d_status);
    }
    ++P->prof->launches[TAPS_PROF_MODEDIAG];   // W^T c
    const long long rm = (long long)Rf * M;
    md_cw_kernel<<<(unsigned)((rm + 255) / 256), 256, 0, s>>>(P->d_c, Wm, Rf, M, cw);
  }
  cudaError_t ce = cudaSuccess;
  switch (hb) {
    case 1: ce = md_band_launch<1>(bx, by, lam, P->d_q[d], cw, Rf, n, M, Ab, scratch, Z, P->d_status, s); break;
    case 2: ce = md_band_launch<2>(bx, by, lam, P->d_q[d], cw, Rf, n, M, Ab, scratch, Z, P->d_status, s); break;
    case 3: ce = md_band_launch<3>(bx, by, lam, P->d_q[d], cw, Rf, n, M, Ab, scratch, Z, P->d_status, s); break;
    case 4: ce = md_band_launch<4>(bx, by, lam, P->d_q[d], cw, Rf, n, M, Ab, scratch, Z, P->d_status, s); break;
    default: ce = md_band_launch<5>(bx, by, lam, P->d_q[d], cw, Rf, n, M, Ab, scratch, Z, P->d_status, s); break;
  }
  TAPS_CUDA(ce);
  const long long nM = (long long)n * M;
  md_out_kernel<<<(unsigned)((nM + 255) / 256), 256, 0, s>>>(Z, Wm, n, M, U->d_U[d], P->d_Uold);
  P->prof->launches[TAPS_PROF_MODEDIAG] += 3;
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

// The eigen-solve of a mode-side solve on its own (exposed so that it can be tested
// against a dense symmetric-definite eigensolver): cold start, 32 < M with S and V in
// shared memory.  Synchronous on `stream`.
extern "C" int taps_util_md_pencil(const double* CX, const double* CY, int M, double* W, double* lam, int* refined,
                                   void* stream) {
  if (!CX || !W || !lam || M <= 32 || M > TAPS_MAX_M) return TAPS_ERR_INVALID_ARG;
  const int Np = M + (M & 1);
  if (sizeof(double) * ((size_t)Np * (Np + 1) + (size_t)M * M) > (size_t)MDB_SMEM_SV_MAX) return TAPS_ERR_INVALID_ARG;
  int dev = 0, maxsm = 0, num_sms = 0;
  TAPS_CUDA(cudaGetDevice(&dev));
  TAPS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  TAPS_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  TAPS_TRY(taps_md_setup(maxsm));
  cudaStream_t s = (cudaStream_t)stream;
  const size_t MM = (size_t)M * M;
  double* gw = nullptr;
  int* dint = nullptr;   // [0] basis mode count (0: cold), [1] status
  TAPS_TRY(taps_alloc((void**)&gw, sizeof(double) * (14 * MM + 8)));
  if (taps_alloc((void**)&dint, 2 * sizeof(int)) != TAPS_OK) {
    cudaFree(gw);
    return TAPS_ERR_CUDA;
  }
  int st = TAPS_OK;
  int h[2] = {0, 0}, acc = 0;
  if (cudaMemsetAsync(dint, 0, 2 * sizeof(int), s) != cudaSuccess) st = TAPS_ERR_CUDA;
  if (st == TAPS_OK) st = md_eig_split(CX, CY, M, W, dint, lam, gw, dint + 1, num_sms, s);
  if (st == TAPS_OK) {
    if (cudaMemcpyAsync(h, dint, 2 * sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&acc, gw + 14 * MM + MR_MAX_STEPS + 1, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      st = TAPS_ERR_CUDA;
  }
  cudaFree(gw);
  cudaFree(dint);
  if (st != TAPS_OK) return st;
  if (h[1] != TAPS_DEV_OK) return taps_status_from_device(h[1]);
  if (refined) *refined = acc;
  return TAPS_OK;
}
