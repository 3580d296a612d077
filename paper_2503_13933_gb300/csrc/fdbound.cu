// Node-side diagonalisation of a dimension with convection faces (Sec. 2.6 route,
// extended to the point-mass terms of Eqs. 21/25).
//
// A space dim with convection faces has, besides its stiffness A (K) and mass B (M or
// W), one or two point-mass operators beta_b e_b e_b^T at its end nodes b.  With the
// pencil basis Phi (Phi^T B Phi = I, Phi^T A Phi = diag(mu)) and U = Phi Y, row i of the
// reduced system reads
//     T_i y_i + sum_b beta_b phi_b[i] C_b z_b = g_i,   z_b = sum_j phi_b[j] y_j,
// with T_i = mu_i C_A + C_B, g_i = (Phi^T F)[i], phi_b = Phi^T e_b (row b of Phi) and
// C_b the coefficient matrix of face b's operator.  The face terms couple the nodes
// only through the nb M-vectors z_b, so (Sherman-Morrison-Woodbury)
//     y_i = w_i - T_i^-1 sum_b beta_b phi_b[i] C_b z_b,   w_i = T_i^-1 g_i,
// and the z_b solve the (nb M) x (nb M) capacitance system
//     z_b' + sum_b beta_b (sum_i phi_b'[i] phi_b[i] T_i^-1) C_b z_b = sum_i phi_b'[i] w_i.
//
//   fdw_node_kernel    warp per node: LU of T_i without pivoting, w_i and T_i^-1
//                      (1 + M right-hand sides, lane = row).
//   fdw_reduce_kernel  the sums over the nodes: Z_b'b = sum_i phi_b' phi_b T_i^-1 and
//                      the capacitance right-hand side.
//   fdw_zc_kernel      the capacitance blocks Z_b'b C_b.
//   fdw_cap_kernel     one CTA: the capacitance system by Gaussian elimination with
//                      partial pivoting, then u_b = C_b z_b.
//   fdw_final_kernel   y_i; then the node-side transform U = Phi Y (fd_rowgemm_kernel).
#include <string.h>

#include <algorithm>

#include "taps_internal.cuh"

// Forward and backward substitution with the warp's LU factors (lane r holds row r:
// unit-lower multipliers left of the diagonal, U on and right of it) for NC
// right-hand-side columns held as rhs[c] in lane r.  invd is 1 / U[r][r] in lane r.
template <int NC>
__device__ __forceinline__ void fdw_warp_solve(const double row[33], double invd, double rhs[NC], int lane,
                                               int M, int ncol) {
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    if (p < M) {
      const double l = row[p];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < ncol) {
          const double v = __shfl_sync(0xffffffffu, rhs[c], p);
          if (lane > p && lane < M) rhs[c] -= l * v;
        }
      }
    }
  }
#pragma unroll
  for (int p = 31; p >= 0; --p) {
    if (p < M) {
      const double u = row[p];
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (c < ncol) {
          if (lane == p) rhs[c] *= invd;
          const double v = __shfl_sync(0xffffffffu, rhs[c], p);
          if (lane < p) rhs[c] -= u * v;
        }
      }
    }
  }
}

__global__ void __launch_bounds__(32) fdw_node_kernel(const double* __restrict__ CA, const double* __restrict__ CB,
                                                      const double* __restrict__ mu, const double* __restrict__ pq,
                                                      const double* __restrict__ c, int Rf, int n, int M,
                                                      double* __restrict__ X, double* __restrict__ w,
                                                      int* status) {
  const int i = blockIdx.x, lane = threadIdx.x;
  const bool act = lane < M;
  const double mi = mu[i];
  double row[33];
#pragma unroll
  for (int k = 0; k < 33; ++k) row[k] = 0.0;
  if (act) {
#pragma unroll
    for (int k = 0; k < 32; ++k)
      if (k < M) row[k] = fma(mi, CA[lane * M + k], CB[lane * M + k]);
  }
  // LU without pivoting: the symmetric part of T_i is positive definite
  bool bad = false;
#pragma unroll
  for (int p = 0; p < 32; ++p) {
    if (p < M) {
      const double piv = __shfl_sync(0xffffffffu, row[p], p);
      bad |= !(fabs(piv) > 0.0) || !isfinite(piv);
      const double ip = (fabs(piv) > 0.0 && isfinite(piv)) ? taps_rcp(piv) : 0.0;
      const double l = (lane > p && act) ? row[p] * ip : 0.0;
#pragma unroll
      for (int k = 0; k < 32; ++k) {
        if (k > p && k < M) {
          const double pk = __shfl_sync(0xffffffffu, row[k], p);
          row[k] -= l * pk;
        }
      }
      if (lane > p && act) row[p] = l;
    }
  }
  if (bad && lane == 0) taps_flag(status, TAPS_DEV_SINGULAR);
  double diag = 1.0;   // U[lane][lane], selected with compile-time register indices
#pragma unroll
  for (int k = 0; k < 32; ++k)
    if (k == lane) diag = row[k];
  const double invd = (act && fabs(diag) > 0.0 && isfinite(diag)) ? taps_rcp(diag) : 0.0;
  // w_i = T_i^-1 g_i, g_i = sum_r pq[r][i] c_r
  double g[1];
  g[0] = 0.0;
  if (act)
    for (int r = 0; r < Rf; ++r) g[0] = fma(pq[(size_t)r * n + i], c[r * M + lane], g[0]);
  fdw_warp_solve<1>(row, invd, g, lane, M, 1);
  if (act) w[(size_t)i * M + lane] = g[0];
  // T_i^-1 (row `lane`, all columns)
  {
    double rhs[32];
#pragma unroll
    for (int k = 0; k < 32; ++k) rhs[k] = (act && k == lane) ? 1.0 : 0.0;
    fdw_warp_solve<32>(row, invd, rhs, lane, M, M);
    if (act) {
      double* out = X + ((size_t)i * M + lane) * M;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (k < M) out[k] = rhs[k];
    }
  }
}

// Z[b'][b][r][c] = sum_i phi_b'[i] phi_b[i] T_i^-1[r][c];  rr[b'][r] = sum_i phi_b'[i] w_i[r].
// phi_b[i] = Phi[corner_b][i] (row corner_b of Phi: Phi^T e_b).  X holds T_i^-1.
__global__ void fdw_reduce_kernel(const double* __restrict__ X, const double* __restrict__ w,
                                  const double* __restrict__ Phi, int c0, int c1, int n, int M, int nbnd,
                                  double* __restrict__ Z, double* __restrict__ rr) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  const int nsc = nbnd * nbnd * M * M;
  if (idx < nsc) {
    const int cc = idx % M, r = (idx / M) % M, b = (idx / (M * M)) % nbnd, bp = idx / (M * M * nbnd);
    const double* pb = Phi + (size_t)(b == 0 ? c0 : c1) * n;
    const double* pbp = Phi + (size_t)(bp == 0 ? c0 : c1) * n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(pbp[i] * pb[i], X[((size_t)i * M + r) * M + cc], s);
    Z[idx] = s;
  } else if (idx < nsc + nbnd * M) {
    const int k = idx - nsc, r = k % M, bp = k / M;
    const double* pbp = Phi + (size_t)(bp == 0 ? c0 : c1) * n;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s = fma(pbp[i], w[(size_t)i * M + r], s);
    rr[k] = s;
  }
}

// SC[b'][b] = Z[b'][b] C_b (M x M products).
__global__ void fdw_zc_kernel(const double* __restrict__ Z, const double* __restrict__ C0,
                              const double* __restrict__ C1, int M, int nbnd, double* __restrict__ SC) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nbnd * nbnd * M * M) return;
  const int cc = idx % M, r = (idx / M) % M, b = (idx / (M * M)) % nbnd;
  const double* Cb = b == 0 ? C0 : C1;
  const double* zr = Z + (size_t)(idx - cc);   // row r of Z[b'][b]
  double s = 0.0;
  for (int k = 0; k < M; ++k) s = fma(zr[k], Cb[(size_t)k * M + cc], s);
  (void)r;
  SC[idx] = s;
}

// (I + [beta_b SC[b'][b]]) z = rr, N2 = nbnd M <= 64 unknowns, partial pivoting; beta_b
// is the corner entry of face b's point-mass band.  Writes u_b = C_b z_b and beta for the
// final kernel.
#define FDW_MAXN 64
__global__ void __launch_bounds__(64) fdw_cap_kernel(const double* __restrict__ SC, const double* __restrict__ rr,
                                                     const double* __restrict__ band0,
                                                     const double* __restrict__ band1, int corner0, int corner1,
                                                     int hb, int M, int nbnd, const double* __restrict__ C0,
                                                     const double* __restrict__ C1, double* __restrict__ z,
                                                     double* __restrict__ beta, int* status) {
  __shared__ double A[FDW_MAXN][FDW_MAXN + 1];
  __shared__ double bet[2];
  __shared__ int piv;
  const int tid = threadIdx.x, N2 = nbnd * M, nb = 2 * hb + 1;
  if (tid < nbnd) {
    const double* bd = tid == 0 ? band0 : band1;
    const int cr = tid == 0 ? corner0 : corner1;
    bet[tid] = bd[(size_t)cr * nb + hb];
  }
  __syncthreads();
  for (int idx = tid; idx < N2 * N2; idx += blockDim.x) {
    const int rI = idx / N2, cI = idx % N2;
    const int bp = rI / M, r = rI % M, b = cI / M, cc = cI % M;
    A[rI][cI] = (rI == cI ? 1.0 : 0.0) + bet[b] * SC[(((size_t)bp * nbnd + b) * M + r) * M + cc];
  }
  for (int rI = tid; rI < N2; rI += blockDim.x) A[rI][N2] = rr[rI];
  if (tid < nbnd) beta[tid] = bet[tid];
  __syncthreads();
  for (int k = 0; k < N2; ++k) {
    if (tid == 0) {
      int best = k;
      double bv = fabs(A[k][k]);
      for (int rI = k + 1; rI < N2; ++rI)
        if (fabs(A[rI][k]) > bv) {
          bv = fabs(A[rI][k]);
          best = rI;
        }
      piv = best;
      if (!(bv > 0.0) || !isfinite(bv)) taps_flag(status, TAPS_DEV_SINGULAR);
    }
    __syncthreads();
    const int pr = piv;
    if (pr != k)
      for (int cI = tid; cI <= N2; cI += blockDim.x) {
        const double t = A[k][cI];
        A[k][cI] = A[pr][cI];
        A[pr][cI] = t;
      }
    __syncthreads();
    const double d = A[k][k];
    const double id = (fabs(d) > 0.0 && isfinite(d)) ? taps_rcp(d) : 0.0;
    for (int rI = k + 1 + tid; rI < N2; rI += blockDim.x) {
      const double l = A[rI][k] * id;
      for (int cI = k + 1; cI <= N2; ++cI) A[rI][cI] -= l * A[k][cI];
    }
    __syncthreads();
  }
  if (tid == 0) {
    for (int k = N2 - 1; k >= 0; --k) {
      double s = A[k][N2];
      for (int cI = k + 1; cI < N2; ++cI) s -= A[k][cI] * A[cI][N2];
      const double d = A[k][k];
      A[k][N2] = (fabs(d) > 0.0 && isfinite(d)) ? s * taps_rcp(d) : 0.0;
    }
  }
  __syncthreads();
  // u_b = C_b z_b, stored in z's place (the final kernel needs only u)
  for (int rI = tid; rI < N2; rI += blockDim.x) {
    const int b = rI / M, r = rI % M;
    const double* Cb = b == 0 ? C0 : C1;
    double u = 0.0;
    for (int k = 0; k < M; ++k) u = fma(Cb[(size_t)r * M + k], A[b * M + k][N2], u);
    z[rI] = u;
  }
}

// Y[i][r] = w_i[r] - (T_i^-1 v_i)[r],  v_i = sum_b beta_b phi_b[i] u_b   (row-major n x M)
__global__ void fdw_final_kernel(const double* __restrict__ X, const double* __restrict__ w,
                                 const double* __restrict__ u, const double* __restrict__ beta,
                                 const double* __restrict__ Phi, int c0, int c1, int n, int M, int nbnd,
                                 double* __restrict__ Y) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * M) return;
  const int r = (int)(idx % M), i = (int)(idx / M);
  const double f0 = beta[0] * Phi[(size_t)c0 * n + i];
  const double f1 = nbnd > 1 ? beta[1] * Phi[(size_t)c1 * n + i] : 0.0;
  const double* x = X + ((size_t)i * M + r) * M;
  double s = 0.0;
  for (int k = 0; k < M; ++k) {
    const double v = nbnd > 1 ? fma(f1, u[M + k], f0 * u[k]) : f0 * u[k];
    s = fma(x[k], v, s);
  }
  Y[idx] = w[idx] - s;
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
int taps_fdw_eligible(const taps_problem* P, int d, int M, int* slotA, int* slotB, int* slotC0, int* slotC1,
                      int* nbnd) {
  const int nops = P->tt.nops[d];
  if (nops < 3 || nops > 4 || M < 1 || M > 32) return 0;
  int a = -1, b = -1, lo = -1, hi = -1;
  for (int s = 0; s < nops; ++s) {
    const int op = P->ops[d][s];
    if (op == TAPS_OP_BLO) {
      if (lo >= 0) return 0;
      lo = s;
    } else if (op == TAPS_OP_BHI) {
      if (hi >= 0) return 0;
      hi = s;
    } else if (op == TAPS_OP_M || op == TAPS_OP_W) {
      if (b >= 0) return 0;
      b = s;
    } else if (op == TAPS_OP_K) {
      if (a >= 0) return 0;
      a = s;
    } else {
      return 0;
    }
  }
  if (a < 0 || b < 0 || (lo < 0 && hi < 0)) return 0;
  *slotA = a;
  *slotB = b;
  *nbnd = 0;
  *slotC0 = *slotC1 = -1;
  if (lo >= 0) *(((*nbnd)++ == 0) ? slotC0 : slotC1) = lo;
  if (hi >= 0) *(((*nbnd)++ == 0) ? slotC0 : slotC1) = hi;
  return 1;
}

// T_i^-1 [nf_max][M][M], w [nf_max][M], Z and SC [4][M][M] each, rr, z / u, beta.
size_t taps_fdw_scratch_doubles(int nf_max, int M) {
  return (size_t)nf_max * ((size_t)M * M + M) + 8 * (size_t)M * M + 4 * (size_t)M + 8;
}

// Reduced solve of dim d (coefficients in P->d_C / P->d_c) through the pencil of its
// stiffness and mass operators; the previous factor goes to P->d_Uold.
int taps_fdw_solve(taps_problem* P, taps_factors* U, int d) {
  int sa, sb, s0, s1, nbnd;
  const int M = U->M;
  if (!taps_fdw_eligible(P, d, M, &sa, &sb, &s0, &s1, &nbnd) || !P->d_fdw || !P->d_pq[d])
    return TAPS_ERR_INVALID_ARG;
  const FdEntry* E = nullptr;
  TAPS_TRY(taps_fd_lookup(P, d, P->ops[d][sa], P->ops[d][sb], &E));
  const taps_dim* dm = P->dims[d];
  const int n = dm->nf, hb = dm->hb;
  const size_t MM = (size_t)M * M;
  cudaStream_t s = P->stream;
  double* X = P->d_fdw;                        // T_i^-1
  double* w = X + (size_t)P->nf_max * MM;
  double* Z = w + (size_t)P->nf_max * M;
  double* SC = Z + 4 * MM;
  double* rr = SC + 4 * MM;
  double* z = rr + 2 * (size_t)M;
  double* beta = z + 2 * (size_t)M;
  double* Y = P->d_Y + (size_t)n * M;
  const int k0 = P->ops[d][s0], k1 = s1 >= 0 ? P->ops[d][s1] : k0;
  const int corner0 = k0 == TAPS_OP_BLO ? 0 : n - 1, corner1 = k1 == TAPS_OP_BLO ? 0 : n - 1;
  const size_t bsz = (size_t)n * dm->nb;
  const double* C0 = P->d_C + (size_t)s0 * MM;
  const double* C1 = s1 >= 0 ? P->d_C + (size_t)s1 * MM : C0;
  int tk = prof_begin(P, TAPS_PROF_FASTDIAG);
  fdw_node_kernel<<<n, 32, 0, s>>>(P->d_C + (size_t)sa * MM, P->d_C + (size_t)sb * MM, E->mu, P->d_pq[d], P->d_c,
                                   P->Rf, n, M, X, w, P->d_status);
  const int nred = nbnd * nbnd * M * M + nbnd * M;
  fdw_reduce_kernel<<<(nred + 127) / 128, 128, 0, s>>>(X, w, E->Phi, corner0, corner1, n, M, nbnd, Z, rr);
  const int nzc = nbnd * nbnd * M * M;
  fdw_zc_kernel<<<(nzc + 127) / 128, 128, 0, s>>>(Z, C0, C1, M, nbnd, SC);
  fdw_cap_kernel<<<1, 64, 0, s>>>(SC, rr, dm->d_band + (size_t)k0 * bsz, dm->d_band + (size_t)k1 * bsz, corner0,
                                  corner1, hb, M, nbnd, C0, C1, z, beta, P->d_status);
  const long long nM = (long long)n * M;
  fdw_final_kernel<<<(unsigned)((nM + 255) / 256), 256, 0, s>>>(X, w, z, beta, E->Phi, corner0, corner1, n, M,
                                                                 nbnd, Y);
  P->prof->launches[TAPS_PROF_FASTDIAG] += 4;
  const double Md = M;
  prof_end(P, TAPS_PROF_FASTDIAG, tk,
           n * ((2.0 / 3.0) * Md * Md * Md + (1.0 + Md) * 2.0 * Md * Md + 2.0 * P->Rf * Md) +
               2.0 * n * (nbnd * nbnd * (double)MM + nbnd * Md) + 2.0 * nbnd * nbnd * (double)MM * Md +
               (2.0 / 3.0) * pow(nbnd * Md, 3) + 2.0 * (double)nM * (Md + nbnd),
           8.0 * ((double)n * MM * 2.0 + 4.0 * nM));
  TAPS_CUDA(cudaGetLastError());
  // back to the nodal basis; the previous factor goes to d_Uold
  return taps_fd_to_nodal(P, E, Y, n, M, U->d_U[d], P->d_Uold);
}
