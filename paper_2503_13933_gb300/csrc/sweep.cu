// Subspace-iteration sweep (Algorithm 1, Eq. 43) on the device: Gram refresh (fused
// banded SpMM + U^T Y, Eq. 34), coefficient combine (Hadamard products over the other
// dimensions, Eq. 35), block-banded reduced system (Eqs. 36-40) and its solve,
// column normalisation and factor change; residuals of Eq. 42 and of the full system.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include <cuda_bf16.h>

#include "taps_internal.cuh"

// ---------------------------------------------------------------------------------
// Coefficients of dim d: C_o = sum_{t: op(t,d) = o} alpha_t prod_{e != d} Gamma_{op(t,e),e}
// and c_r = beta_r prod_{e != d} h_{r,e} (Eq. 35), entry idx of the M x M matrices.
// ---------------------------------------------------------------------------------
// The loads of one product are issued together (unrolled over TAPS_MAX_DIMS, predicated
// off for the skipped dims) so that their latencies overlap; the product then multiplies
// only the D - 1 real factors in increasing dim order (each FP64 instruction holds the
// pipe ~64 cycles on this GPU, so the exact multiplications by 1 of unused dim slots
// and an add per possible operator slot were most of the work).  Each operator slot's
// sum takes its terms in increasing order.
// More distinct operators than TAPS_NUM_OPS (weighted operators): one slot at a time,
// the terms in the same order, so each slot's sum is the one the register version forms.
__device__ __forceinline__ void coeff_C_slots(const TermTable& tt, const GramPtrs& gp, int d, int M, int idx,
                                           double* C) {
  const int MM = M * M;
  for (int o = 0; o < tt.nops[d]; ++o) {
    double acc = 0.0;
    for (int t = 0; t < tt.R; ++t) {
      if (tt.oi[t][d] != o) continue;
      double prod = tt.alpha[t];
      for (int e = 0; e < tt.D; ++e)
        if (e != d) prod *= __ldcg(gp.gram[e] + (size_t)tt.oi[t][e] * MM + idx);
      acc += prod;
    }
    C[(size_t)o * MM + idx] = acc;
  }
}

__device__ __forceinline__ void coeff_C(const TermTable& tt, const GramPtrs& gp, int d, int M, int idx,
                                        double* C) {
  const int MM = M * M;
  for (int o = 0; o < tt.nops[d]; ++o) {
    double acc = 0.0;
    for (int t = 0; t < tt.R; ++t) {
      if (tt.oi[t][d] != o) continue;
      double f[TAPS_MAX_DIMS];
#pragma unroll
      for (int e = 0; e < TAPS_MAX_DIMS; ++e)
        f[e] = (e < tt.D && e != d) ? __ldcg(gp.gram[e] + (size_t)tt.oi[t][e] * MM + idx) : 1.0;
      double prod = tt.alpha[t];
#pragma unroll
      for (int e = 0; e < TAPS_MAX_DIMS; ++e)
        if (e < tt.D && e != d) prod *= f[e];
      acc += prod;
    }
    C[(size_t)o * MM + idx] = acc;
  }
}

__device__ __forceinline__ void coeff_c(const TermTable& tt, const GramPtrs& gp, int d, int M, int r, int m,
                                        double* c) {
  double f[TAPS_MAX_DIMS];
#pragma unroll
  for (int e = 0; e < TAPS_MAX_DIMS; ++e)
    f[e] = (e < tt.D && e != d) ? __ldcg(gp.h[e] + (size_t)r * M + m) : 1.0;
  double v = tt.beta[r];
#pragma unroll
  for (int e = 0; e < TAPS_MAX_DIMS; ++e)
    if (e < tt.D && e != d) v *= f[e];
  c[(size_t)r * M + m] = v;
}

__device__ __forceinline__ void coeff_entry(const TermTable& tt, const GramPtrs& gp, int d, int M, int idx,
                                            double* C, double* c) {
  if (idx < M * M) coeff_C(tt, gp, d, M, idx, C);
  if (idx < tt.Rf * M) coeff_c(tt, gp, d, M, idx / M, idx % M, c);   // one thread per (r, m)
}

__global__ void coeff_kernel(TermTable tt, GramPtrs gp, int d, int M, double* C, double* c) {
  taps_pdl_wait();
  coeff_entry(tt, gp, d, M, blockIdx.x * blockDim.x + threadIdx.x, C, c);
}

// Coefficients of every dim at once (blockIdx.y = dim), into [D][TAPS_NUM_OPS][M][M]
// and [D][Rf][M].
__global__ void coeff_all_kernel(TermTable tt, GramPtrs gp, int M, double* Call, double* call) {
  taps_pdl_wait();
  const int d = blockIdx.y;
  coeff_entry(tt, gp, d, M, blockIdx.x * blockDim.x + threadIdx.x,
              Call + (size_t)d * TAPS_NUM_OPS * M * M, call + (size_t)d * tt.Rf * M);
}

// The same with more distinct operators than TAPS_NUM_OPS in some dim (weighted
// operators): coefficient arrays with slot stride tt.cs.
__device__ __forceinline__ void coeff_entry_slots(const TermTable& tt, const GramPtrs& gp, int d, int M, int idx,
                                                  double* C, double* c) {
  if (idx < M * M) coeff_C_slots(tt, gp, d, M, idx, C);
  if (idx < tt.Rf * M) coeff_c(tt, gp, d, M, idx / M, idx % M, c);   // one thread per (r, m)
}

__global__ void coeff_slots_kernel(TermTable tt, GramPtrs gp, int d, int M, double* C, double* c) {
  taps_pdl_wait();
  coeff_entry_slots(tt, gp, d, M, blockIdx.x * blockDim.x + threadIdx.x, C, c);
}

__global__ void coeff_all_slots_kernel(TermTable tt, GramPtrs gp, int M, double* Call, double* call) {
  taps_pdl_wait();
  const int d = blockIdx.y;
  coeff_entry_slots(tt, gp, d, M, blockIdx.x * blockDim.x + threadIdx.x,
                    Call + (size_t)d * tt.cs * M * M, call + (size_t)d * tt.Rf * M);
}

// ---------------------------------------------------------------------------------
// Gram refresh of one dimension: Gamma_o = U^T Op_o U for each distinct op o and
// h_r = U^T q_r (Eq. 34).  CTA (chunk, mtile) handles GR rows and MT rows of Gamma and
// writes its partial sums; per mode tile the last CTA to finish (a ticket counter, no
// waiting) sums the tile's partials in a fixed chunk order and, when asked, forms
// the tile's rows of the next dimension's coefficients from the fresh Grams, so one
// launch does all three steps.
// ---------------------------------------------------------------------------------
#define GR 8

// Operand as the contraction sees it: with BF16IN rounded to bfloat16 (round to
// nearest even) and widened to the accumulation type.
template <typename T, bool BF16IN>
__device__ __forceinline__ T gram_in(double x) {
  if (BF16IN) return (T)__bfloat162float(__float2bfloat16_rn((float)x));
  return (T)x;
}

template <typename T, bool BF16IN>
__device__ __forceinline__ void gram_partial_body(int chunk, int tile, int nchunk, const double* __restrict__ U,
                                                  int nf, int M, int hb, const double* __restrict__ opband,
                                                  int nops, const double* __restrict__ q, int Rf,
                                                  double* __restrict__ partial, int stride, unsigned* ticket,
                                                  double* gram, double* h, const TermTable& tt,
                                                  const GramPtrs& gp, int cd, double* C, double* c, int gmt,
                                                  int tail) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int is_last;
  const int nb = 2 * hb + 1;
  const int rows_h = GR + 2 * hb;
  T* Us = reinterpret_cast<T*>(smem_raw);  // [rows_h][M]
  T* Ys = Us + rows_h * M;                 // [GR][M]
  T* Bs = Ys + GR * M;                     // [nops][GR][nb] the chunk's band rows
  T* Qs = Bs + nops * GR * nb;             // [Rf][GR] the chunk's source rows
  const int r0 = chunk * GR;
  const int m0 = tile * gmt;
  const int mt = min(gmt, M - m0);
  taps_pdl_wait();
  // the factor rows, band rows and source rows of the chunk in one load phase, so that
  // the products below read shared memory only
  for (int idx = threadIdx.x; idx < rows_h * M; idx += blockDim.x) {
    int m = idx / rows_h, rr = idx % rows_h;
    int gi = r0 - hb + rr;
    Us[rr * M + m] = (gi >= 0 && gi < nf) ? gram_in<T, BF16IN>(U[(size_t)m * nf + gi]) : (T)0;
  }
  for (int idx = threadIdx.x; idx < nops * GR * nb; idx += blockDim.x) {
    const int o = idx / (GR * nb), rem = idx % (GR * nb);
    const int gi = r0 + rem / nb;
    Bs[idx] = gi < nf ? gram_in<T, BF16IN>(opband[((size_t)o * nf + gi) * nb + rem % nb]) : (T)0;
  }
  for (int idx = threadIdx.x; idx < Rf * GR; idx += blockDim.x) {
    const int r = idx / GR, gi = r0 + idx % GR;
    Qs[idx] = gi < nf ? gram_in<T, BF16IN>(q[(size_t)r * nf + gi]) : (T)0;
  }
  __syncthreads();
  double* out = partial + ((size_t)chunk) * stride;
  for (int o = 0; o < nops; ++o) {
    for (int idx = threadIdx.x; idx < GR * M; idx += blockDim.x) {
      int i = idx / M, n = idx % M;
      int gi = r0 + i;
      T acc = 0;
      if (gi < nf) {
        const T* brow = Bs + (o * GR + i) * nb;
        for (int k = 0; k < nb; ++k) acc += brow[k] * Us[(i + k) * M + n];
      }
      Ys[i * M + n] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < mt * M; idx += blockDim.x) {
      int m = m0 + idx / M, n = idx % M;
      T acc = 0;
      for (int i = 0; i < GR; ++i) acc += Us[(i + hb) * M + m] * Ys[i * M + n];
      out[((size_t)o * M + m) * M + n] = (double)acc;
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < Rf * mt; idx += blockDim.x) {
    int r = idx / mt, m = m0 + idx % mt;
    T acc = 0;
    for (int i = 0; i < GR; ++i) {
      int gi = r0 + i;
      if (gi < nf) acc += Qs[r * GR + i] * Us[(i + hb) * M + m];
    }
    out[(size_t)nops * M * M + (size_t)r * M + m] = (double)acc;
  }
  if (!tail) return;   // gram_reduce_coeff_kernel adds the partials
  // ---- per mode tile, the last chunk CTA reduces the tile's slice of the partials
  // and forms the tile's rows of the coefficients of dim cd.  Ticket y counts the
  // CTAs of tile y.
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(ticket + tile, 1u) == (unsigned)(nchunk - 1)) ? 1 : 0;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
    const int ng = nops * M * M;
  const int nslice = nops * mt * M + Rf * mt;   // this tile's rows of every Gamma_o, then of h
  for (int e = threadIdx.x; e < nslice; e += blockDim.x) {
    int j;
    if (e < nops * mt * M) {
      const int o = e / (mt * M), rem = e % (mt * M);
      j = (o * M + m0 + rem / M) * M + rem % M;
    } else {
      const int rem = e - nops * mt * M;
      j = ng + (rem / mt) * M + m0 + rem % mt;
    }
    // chunk partials 32 at a time: the loads of a batch in flight together, then the
    // sum in chunk order
    double acc = 0.0;
    for (int c0 = 0; c0 < nchunk; c0 += 32) {
      double v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = (c0 + k < nchunk) ? __ldcg(partial + (size_t)(c0 + k) * stride + j) : 0.0;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (c0 + k < nchunk) acc += v[k];
    }
    if (j < ng) gram[j] = acc;
    else h[j - ng] = acc;
  }
  if (threadIdx.x == 0) ticket[tile] = 0u;   // ready for the next launch on this stream
  if (cd < 0) return;
  // entry (m, n) of the coefficients needs entry (m, n) of each dim's Gram only, so
  // this CTA forms the rows m of its tile (the Gram rows it just wrote are visible to
  // its threads after the barrier); the matrix and source entries in one pass
  __syncthreads();
  for (int e = threadIdx.x; e < mt * M + Rf * mt; e += blockDim.x) {
    if (e < mt * M) coeff_C(tt, gp, cd, M, m0 * M + e, C);
    else coeff_c(tt, gp, cd, M, (e - mt * M) / mt, m0 + (e - mt * M) % mt, c);
  }
}

template <typename T, bool BF16IN>
__global__ void gram_partial_kernel(const double* __restrict__ U, int nf, int M, int hb,
                                    const double* __restrict__ opband, int nops,
                                    const double* __restrict__ q, int Rf,
                                    double* __restrict__ partial, int stride, unsigned* ticket,
                                    double* gram, double* h, TermTable tt, GramPtrs gp, int cd,
                                    double* C, double* c, int gmt, int tail) {
  gram_partial_body<T, BF16IN>(blockIdx.x, blockIdx.y, gridDim.x, U, nf, M, hb, opband, nops, q, Rf, partial,
                               stride, ticket, gram, h, tt, gp, cd, C, c, gmt, tail);
}

// The chunk partials of a dim's Grams added in chunk order and the next dim's
// coefficients, spread over many small CTAs: CTA b < ceil(M^2 / 32) takes the 32 entries
// (m, n) = 32b .. 32b+31, warp w adds entries (o, m, n) of Gamma_o, o = w, w + 8, ...,
// over the chunks (32 partials in flight at a time; at most eight warps), and after
// the block barrier warp 0 forms C(m, n) of dim
// cd from them; the CTAs after those add the source projections h_r[m] and form c.  The
// same sums and coefficient functions as the last-CTA tail of gram_partial_kernel, whose
// FP64 work ran on one SM per mode tile.
__global__ void gram_reduce_coeff_kernel(const double* __restrict__ partial, int stride, int nchunk, int M,
                                         int nops, int Rf, double* gram, double* h, TermTable tt, GramPtrs gp,
                                         int cd, double* C, double* c) {
  taps_pdl_wait();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int MM = M * M, ng = nops * MM;
  const int nCg = (MM + 31) / 32;
  auto chunk_sum = [&](int j) {
    double acc = 0.0;
    for (int c0 = 0; c0 < nchunk; c0 += 32) {
      double v[32];
#pragma unroll
      for (int k = 0; k < 32; ++k) v[k] = (c0 + k < nchunk) ? __ldcg(partial + (size_t)(c0 + k) * stride + j) : 0.0;
#pragma unroll
      for (int k = 0; k < 32; ++k)
        if (c0 + k < nchunk) acc += v[k];
    }
    return acc;
  };
  if ((int)blockIdx.x < nCg) {
    const int idx = blockIdx.x * 32 + lane;
    if (idx < MM)
      for (int o = w; o < nops; o += blockDim.x >> 5) gram[o * MM + idx] = chunk_sum(o * MM + idx);
    __syncthreads();
    if (cd >= 0 && w == 0 && idx < MM) coeff_C(tt, gp, cd, M, idx, C);
  } else {
    const int e = (blockIdx.x - nCg) * 32 + lane;
    if (w == 0 && e < Rf * M) {
      h[e] = chunk_sum(ng + e);
      if (cd >= 0) coeff_c(tt, gp, cd, M, e / M, e % M, c);
    }
  }
}

// The Gram refresh of every dim in one launch (the refresh that starts a solve): CTA
// blockIdx.x is (dim d, mode tile, row chunk) with the same work, partial layout, ticket
// protocol and fixed-order tail sum as gram_partial_kernel's CTA (chunk, tile) of dim d,
// each dim with its own partial region and tickets.
struct GramAll {
  const double* U[TAPS_MAX_DIMS];
  const double* band[TAPS_MAX_DIMS];
  const double* q[TAPS_MAX_DIMS];
  double* partial[TAPS_MAX_DIMS];
  unsigned* ticket[TAPS_MAX_DIMS];
  double* gram[TAPS_MAX_DIMS];
  double* h[TAPS_MAX_DIMS];
  int nf[TAPS_MAX_DIMS], hb[TAPS_MAX_DIMS], nops[TAPS_MAX_DIMS], nchunk[TAPS_MAX_DIMS];
  int cta0[TAPS_MAX_DIMS + 1];
  int D;
};

__global__ void gram_partial_all_kernel(GramAll ga, int M, int Rf, TermTable tt, GramPtrs gp, int gmt) {
  int d = 0;
  while (d + 1 < ga.D && (int)blockIdx.x >= ga.cta0[d + 1]) ++d;
  const int loc = blockIdx.x - ga.cta0[d];
  const int nchunk = ga.nchunk[d];
  const int nops = ga.nops[d];
  gram_partial_body<double, false>(loc % nchunk, loc / nchunk, nchunk, ga.U[d], ga.nf[d], M, ga.hb[d], ga.band[d],
                                   nops, ga.q[d], Rf, ga.partial[d], nops * M * M + Rf * M, ga.ticket[d],
                                   ga.gram[d], ga.h[d], tt, gp, -1, nullptr, nullptr, gmt, 1);
}

// Mode tiles of gmt rows: each tile's last CTA adds its rows' chunk partials, so smaller
// tiles spread that FP64 work over more SMs while every CTA still forms the whole banded
// product of its chunk; 4 rows measured fastest up to 32 modes (8 beyond).  The tile
// height changes no sum's order.  At most 32 tiles (M <= 128).
static int gram_tile_rows(int M) { return M <= 32 ? 4 : 8; }

static GramPtrs gram_ptrs(const taps_problem* P) {
  GramPtrs gp;
  memset(&gp, 0, sizeof(gp));
  for (int d = 0; d < P->D; ++d) {
    gp.gram[d] = P->d_gram[d];
    gp.h[d] = P->d_h[d];
  }
  return gp;
}

static int coefficients(taps_problem* P, int d, int M);
// ---------------------------------------------------------------------------------
// Gram refresh of a long dim with many modes (FP64; M > 32, n >= 256): the banded
// products Y_o = Op_o U once for the whole dim (spmm_kernel), then W = U^T [Y_0 | ... |
// Q] (Q the n x R_f source projections) as a tiled contraction over the nodes: CTA
// (row chunk, 32 x 32 output tile) accumulates KC nodes of its tile (8 x 32 threads,
// four outputs each, operands staged 32 nodes at a time), its partial goes to the
// workspace, and gram_gemm_reduce_kernel adds the chunks' partials in chunk order.
// Every mode tile no longer rebuilds the banded products, and the reduction is over
// n / KC chunks instead of n / 8.
// ---------------------------------------------------------------------------------
#define GG_KC 256
__global__ void spmm_kernel(const double* __restrict__ U, int nf, int M, int hb,
                            const double* __restrict__ opband, int nops, double* __restrict__ Y);
__global__ void __launch_bounds__(256) gram_gemm_kernel(const double* __restrict__ U, int nf, int M,
                                                        const double* __restrict__ Y, int nops,
                                                        const double* __restrict__ q, int Rf,
                                                        double* __restrict__ partial) {
  __shared__ double Us[32][33], Bs[32][33];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int ncol = nops * M + Rf;
  const int ntc = (ncol + 31) / 32;
  const int tm = blockIdx.y / ntc, tc = blockIdx.y % ntc;
  const int m0 = tm * 32, c0 = tc * 32;
  const int k0 = blockIdx.x * GG_KC, k1 = min(nf, k0 + GG_KC);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int kb = k0; kb < k1; kb += 32) {
    // U rows kb.. (node index fastest: coalesced in the column-major factor)
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int mm = e >> 5, kk = e & 31;
      const int i = kb + kk, m = m0 + mm;
      Us[kk][mm] = (i < k1 && m < M) ? U[(size_t)m * nf + i] : 0.0;
    }
    // B columns c0..: Y_o (row-major, column fastest) or Q (node fastest)
    for (int e = threadIdx.x; e < 32 * 32; e += 256) {
      const int kk = e >> 5, cc = e & 31;
      const int i = kb + kk, c = c0 + cc;
      if (c >= nops * M && c < ncol) continue;   // source columns: the loop below
      double v = 0.0;
      if (i < k1 && c < nops * M) {
        const int o = c / M, n = c - o * M;
        v = Y[((size_t)o * nf + i) * M + n];
      }
      Bs[kk][cc] = v;
    }
    if (c0 + 31 >= nops * M) {   // the tile reaches the source columns
      for (int e = threadIdx.x; e < 32 * 32; e += 256) {
        const int cc = e >> 5, kk = e & 31;
        const int i = kb + kk, c = c0 + cc;
        if (c >= nops * M && c < ncol) Bs[kk][cc] = (i < k1) ? q[(size_t)(c - nops * M) * nf + i] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const double b = Bs[kk][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] = fma(Us[kk][ty + 8 * j], b, acc[j]);
    }
    __syncthreads();
  }
  double* out = partial + (size_t)blockIdx.x * M * ncol;
  const int c = c0 + tx;
  if (c < ncol)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int m = m0 + ty + 8 * j;
      if (m < M) out[(size_t)m * ncol + c] = acc[j];
    }
}

// gram[o][m][n] and h[r][m] from the chunks' partials W[m][col], added in chunk order.
__global__ void gram_gemm_reduce_kernel(const double* __restrict__ partial, int nchunk, int M, int nops, int Rf,
                                        double* __restrict__ gram, double* __restrict__ h) {
  const int ncol = nops * M + Rf;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)M * ncol) return;
  const int m = (int)(e / ncol), c = (int)(e % ncol);
  double s = 0.0;
  for (int ch = 0; ch < nchunk; ++ch) s += partial[(size_t)ch * M * ncol + e];
  if (c < nops * M) {
    const int o = c / M, n = c - o * M;
    gram[((size_t)o * M + m) * M + n] = s;
  } else {
    h[(size_t)(c - nops * M) * M + m] = s;
  }
}


int taps_refresh_gram_dim(taps_problem* P, const taps_factors* U, int d, int precision, int coeff_dim) {
  P->c0_valid = 0;   // the Grams of dim d change; the routes below re-form coeff_dim's
  if (P->tt.cs > TAPS_NUM_OPS && coeff_dim >= 0) {
    // weighted operators: the Gram refresh, then the coefficients in their own launch
    TAPS_TRY(taps_refresh_gram_dim(P, U, d, precision, -1));
    const int M = U->M;
    int tk = prof_begin(P, TAPS_PROF_COEFF);
    TAPS_CUDA(taps_launch_pdl(coeff_slots_kernel, dim3((std::max(M * M, P->Rf * M) + 127) / 128), dim3(128), 0, P->stream, P->tt,
                              gram_ptrs(P), coeff_dim, M, P->d_C, P->d_c));
    prof_end(P, TAPS_PROF_COEFF, tk, (double)P->R * M * M * P->D, 8.0 * ((double)P->R * M * M * P->D));
    P->c0_valid = (coeff_dim == 0);
    P->c0_M = M;
    return TAPS_OK;
  }
  const taps_dim* dm = P->dims[d];
  int M = U->M, nf = dm->nf, hb = dm->hb, nops = P->tt.nops[d], Rf = P->Rf;
  if (M == 0) return TAPS_OK;
  int nchunk = (nf + GR - 1) / GR;
  int stride = nops * M * M + Rf * M;
  const int gmt = gram_tile_rows(M);
  dim3 grid(nchunk, (M + gmt - 1) / gmt);
  size_t elems = (size_t)(GR + 2 * hb) * M + (size_t)GR * M + (size_t)nops * GR * (2 * hb + 1) + (size_t)Rf * GR;
  const int nb = 2 * hb + 1;
  double gflops = nops * (2.0 * nb * nf * M + 2.0 * nf * (double)M * M) + 2.0 * Rf * nf * M;
  double gbytes = 8.0 * ((double)nf * M + (double)nops * nf * nb + (double)Rf * nf +
                         (double)nops * M * M + (double)Rf * M);
  if (coeff_dim >= 0) {
    gflops += (double)P->R * M * M * P->D + (double)P->Rf * M * P->D;
    gbytes += 8.0 * ((double)P->R * M * M * P->D);
  }
  GramPtrs gp = gram_ptrs(P);
  if (precision == TAPS_BF16 && taps_gram_tc_eligible(M, nops, Rf, hb)) {
    // BF16 operands on the tensor cores (chunks of 64 nodes, one CTA each), then the
    // next dim's coefficients in their own launch
    int tk = prof_begin(P, TAPS_PROF_GRAM);
    TAPS_TRY(taps_gram_tc_single(U->d_U[d], P->d_opband[d], P->d_q[d], P->d_gram[d], P->d_h[d], nf, M, hb, nops,
                                 Rf, P->d_partial, P->d_ticket + 48, 64, P->stream, P->d_status));
    prof_end(P, TAPS_PROF_GRAM, tk, nops * (2.0 * nb * nf * M + 2.0 * nf * (double)M * M) + 2.0 * Rf * nf * M,
             8.0 * ((double)nf * M + (double)nops * nf * nb + (double)Rf * nf + (double)nops * M * M +
                    (double)Rf * M));
    TAPS_CUDA(cudaGetLastError());
    if (coeff_dim >= 0) TAPS_TRY(coefficients(P, coeff_dim, M));
    return TAPS_OK;
  }
  if (precision != TAPS_FP32 && precision != TAPS_BF16 && M > 32 && nf >= 256 &&
      (size_t)((nf + GG_KC - 1) / GG_KC) * M * (nops * M + Rf) <= P->partial_len) {
    // long dim, many modes: banded products once, then the tiled contraction
    int tk = prof_begin(P, TAPS_PROF_GRAM);
    const long long ny = (long long)nops * nf * M;
    spmm_kernel<<<(unsigned)((ny + 255) / 256), 256, 0, P->stream>>>(U->d_U[d], nf, M, hb, P->d_opband[d], nops,
                                                                     P->d_Y);
    const int ncol = nops * M + Rf;
    const int nkc = (nf + GG_KC - 1) / GG_KC;
    gram_gemm_kernel<<<dim3(nkc, ((M + 31) / 32) * ((ncol + 31) / 32)), 256, 0, P->stream>>>(
        U->d_U[d], nf, M, P->d_Y, nops, P->d_q[d], Rf, P->d_partial);
    const long long nout = (long long)M * ncol;
    gram_gemm_reduce_kernel<<<(unsigned)((nout + 255) / 256), 256, 0, P->stream>>>(P->d_partial, nkc, M, nops, Rf,
                                                                                   P->d_gram[d], P->d_h[d]);
    P->prof->launches[TAPS_PROF_GRAM] += 2;
    prof_end(P, TAPS_PROF_GRAM, tk, gflops - (coeff_dim >= 0 ? (double)P->R * M * M * P->D + (double)P->Rf * M * P->D : 0.0),
             gbytes);
    TAPS_CUDA(cudaGetLastError());
    if (coeff_dim >= 0) TAPS_TRY(coefficients(P, coeff_dim, M));
    return TAPS_OK;
  }
  int tk = prof_begin(P, TAPS_PROF_GRAM);
  if (precision == TAPS_FP32) {   // TAPS_MIXED keeps FP64 Grams
    TAPS_CUDA(taps_launch_pdl(gram_partial_kernel<float, false>, grid, dim3(256), elems * sizeof(float),
                              P->stream, (const double*)U->d_U[d], nf, M, hb, (const double*)P->d_opband[d], nops,
                              (const double*)P->d_q[d], Rf, P->d_partial, stride, P->d_ticket, P->d_gram[d],
                              P->d_h[d], P->tt, gp, coeff_dim, P->d_C, P->d_c, gmt, 1));
  } else if (precision == TAPS_BF16) {
    TAPS_CUDA(taps_launch_pdl(gram_partial_kernel<float, true>, grid, dim3(256), elems * sizeof(float),
                              P->stream, (const double*)U->d_U[d], nf, M, hb, (const double*)P->d_opband[d], nops,
                              (const double*)P->d_q[d], Rf, P->d_partial, stride, P->d_ticket, P->d_gram[d],
                              P->d_h[d], P->tt, gp, coeff_dim, P->d_C, P->d_c, gmt, 1));
  } else {
    // FP64: the chunk partials (8-mode tiles: without the tail, fewer tiles recompute
    // the banded products fewer times), then the chunk sums and coefficients spread over
    // many CTAs
    const int gmt8 = 8;
    TAPS_CUDA(taps_launch_pdl(gram_partial_kernel<double, false>, dim3(nchunk, (M + gmt8 - 1) / gmt8), dim3(256),
                              elems * sizeof(double), P->stream, (const double*)U->d_U[d], nf, M, hb,
                              (const double*)P->d_opband[d], nops, (const double*)P->d_q[d], Rf, P->d_partial, stride,
                              P->d_ticket, P->d_gram[d], P->d_h[d], P->tt, gp, coeff_dim, P->d_C, P->d_c, gmt8, 0));
    const int nCg = (M * M + 31) / 32, nCh = (Rf * M + 31) / 32;
    TAPS_CUDA(taps_launch_pdl(gram_reduce_coeff_kernel, dim3(nCg + nCh), dim3(32 * std::min(nops, 8)), 0, P->stream,
                              (const double*)P->d_partial, stride, nchunk, M, nops, Rf, P->d_gram[d], P->d_h[d],
                              P->tt, gp, coeff_dim, P->d_C, P->d_c));
    P->prof->launches[TAPS_PROF_GRAM] += 1;
  }
  prof_end(P, TAPS_PROF_GRAM, tk, gflops, gbytes);
  TAPS_CUDA(cudaGetLastError());
  P->c0_valid = (coeff_dim == 0);   // the last CTA of each mode tile formed them
  P->c0_M = M;
  return TAPS_OK;
}

// Every dim's Grams; the last refresh also forms dim 0's coefficients for the next sweep.
// In FP64 with every dim on the chunked route (and the partial regions of all dims in
// the workspace), one launch refreshes all dims and a second forms dim 0's coefficients.
int taps_refresh_grams(taps_problem* P, const taps_factors* U, int precision) {
  const int M = U->M;
  bool all = P->gram_all_ok && M >= 1 && (precision == TAPS_FP64 || precision == TAPS_MIXED) &&
             P->tt.cs <= TAPS_NUM_OPS;
  for (int d = 0; d < P->D && all; ++d)
    if (M > 32 && P->dims[d]->nf >= 256) all = false;   // the banded-product + contraction route
  if (!all) {
    for (int d = 0; d < P->D; ++d) TAPS_TRY(taps_refresh_gram_dim(P, U, d, precision, d == P->D - 1 ? 0 : -1));
    return TAPS_OK;
  }
  P->c0_valid = 0;
  const int gmt = gram_tile_rows(M), ntile = (M + gmt - 1) / gmt, Rf = P->Rf;
  GramAll ga;
  memset(&ga, 0, sizeof(ga));
  ga.D = P->D;
  size_t off = 0, elems = 0;
  double gflops = 0.0, gbytes = 0.0;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    const int nf = dm->nf, hb = dm->hb, nops = P->tt.nops[d], nb = 2 * hb + 1;
    ga.U[d] = U->d_U[d];
    ga.band[d] = P->d_opband[d];
    ga.q[d] = P->d_q[d];
    ga.partial[d] = P->d_partial + off;
    ga.ticket[d] = P->d_ticket_all + (size_t)d * 32;
    ga.gram[d] = P->d_gram[d];
    ga.h[d] = P->d_h[d];
    ga.nf[d] = nf;
    ga.hb[d] = hb;
    ga.nops[d] = nops;
    ga.nchunk[d] = (nf + GR - 1) / GR;
    ga.cta0[d + 1] = ga.cta0[d] + ga.nchunk[d] * ntile;
    off += (size_t)ga.nchunk[d] * (nops * M * M + Rf * M);
    elems = std::max(elems, (size_t)(GR + 2 * hb) * M + (size_t)GR * M + (size_t)nops * GR * nb + (size_t)Rf * GR);
    gflops += nops * (2.0 * nb * nf * M + 2.0 * nf * (double)M * M) + 2.0 * Rf * nf * M;
    gbytes += 8.0 * ((double)nf * M + (double)nops * nf * nb + (double)Rf * nf + (double)nops * M * M +
                     (double)Rf * M);
  }
  int tk = prof_begin(P, TAPS_PROF_GRAM);
  TAPS_CUDA(taps_launch_pdl(gram_partial_all_kernel, dim3(ga.cta0[P->D]), dim3(256), elems * sizeof(double),
                            P->stream, ga, M, Rf, P->tt, gram_ptrs(P), gmt));
  prof_end(P, TAPS_PROF_GRAM, tk, gflops, gbytes);
  TAPS_CUDA(cudaGetLastError());
  return coefficients(P, 0, M);
}

// Block band of the reduced matrix (node-major, I = (i, m)):
// block(i, i+k-hb)[m][n] = sum_o Op_o[i, i+k-hb] C_o[m][n]; and F[i][m] = sum_r q_r[i] c_r[m].
__global__ void block_assemble_kernel(const double* __restrict__ opband, int nops, int nf, int nb,
                                      int M, const double* __restrict__ C,
                                      const double* __restrict__ q, const double* __restrict__ c,
                                      int Rf, double* __restrict__ blocks, double* __restrict__ F) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long MM = (long long)M * M;
  long long nblk = (long long)nf * nb * MM;
  if (idx < nblk) {
    long long ik = idx / MM;
    int mn = idx % MM;
    int i = ik / nb, k = ik % nb;
    double v = 0.0;
    for (int o = 0; o < nops; ++o)
      v += opband[((size_t)o * nf + i) * nb + k] * C[(size_t)o * MM + mn];
    blocks[idx] = v;
  } else if (idx < nblk + (long long)nf * M) {
    long long j = idx - nblk;
    int i = j / M, m = j % M;
    double v = 0.0;
    for (int r = 0; r < Rf; ++r) v += q[(size_t)r * nf + i] * c[(size_t)r * M + m];
    F[j] = v;
  }
}

// ---------------------------------------------------------------------------------
// Block-banded Gaussian elimination without pivoting (one cooperative launch).
// For each block row k: every CTA that has solve work factors the diagonal block
// D_k = A(k,k) = L U in its own shared memory (no barrier, no global copy), then its
// warps form W_kj = D_k^{-1} A_kj and z_k = D_k^{-1} F_k (one warp per column,
// triangular solves by shuffles); after a grid barrier all threads apply the Schur
// updates A_ij -= A_ik W_kj, F_i -= A_ik z_k; a second barrier closes the row.  The
// factorisation: at step p warp 0 updates row p+1 and takes the next pivot's
// reciprocal (seed plus refinement, within one ulp of the quotient) while warps 1 ..
// update the other rows four at a time, one FMA per entry (lanes over the columns), so
// the pivot chain is the step's only serial part; the reciprocals are kept for the
// back substitution.  A per-warp triangular solve issues FP64 work only for the
// register slots that hold rows.  Measured phase costs (n = 254, hb = 3, M = 30,
// synthetic blocks): grid barrier ~2.1 µs; per row before these changes LU 27.8 µs,
// triangular solves 20.8 µs.  The
// symmetric part of every reduced matrix is positive definite (Hadamard products of
// Gram matrices, Kronecker products with SPD 1D matrices), so elimination without
// pivoting exists; a zero or non-finite pivot is reported as TAPS_DEV_SINGULAR.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ double slot_get(const double v[4], int s) {
  return s == 0 ? v[0] : (s == 1 ? v[1] : (s == 2 ? v[2] : v[3]));
}
__device__ __forceinline__ void slot_set(double v[4], int s, double x) {
  if (s == 0) v[0] = x;
  else if (s == 1) v[1] = x;
  else if (s == 2) v[2] = x;
  else v[3] = x;
}

__global__ void __launch_bounds__(256) block_lu_kernel(double* __restrict__ blocks,
                                                       double* __restrict__ F,
                                                       double* __restrict__ lu_g, int nf, int hb,
                                                       int M, int* status, unsigned* bar) {
  extern __shared__ __align__(16) double sm[];  // LU of the diagonal block, stride M+1
  __shared__ double invd[TAPS_MAX_M];            // reciprocals of the pivots
  const int nb = 2 * hb + 1;
  const int ld = M + 1;
  const size_t MM = (size_t)M * M;
  const unsigned nblk = gridDim.x;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nthr >> 5;
  const long long gtid = (long long)blockIdx.x * nthr + tid;
  const long long gthreads = (long long)nblk * nthr;
  (void)lu_g;
#define BLK(i, j) (blocks + ((size_t)(i) * nb + ((j) - (i) + hb)) * MM)

  for (int k = 0; k < nf; ++k) {
    const int nj = min(hb, nf - 1 - k);
    const int ntask = nj * M + 1;
    const int cta_needed = (ntask + nwarps - 1) / nwarps;
    if ((int)blockIdx.x < cta_needed) {
      // ---- LU of the diagonal block A(k,k) in this CTA's shared memory
      const double* Akk = BLK(k, k);
      for (int idx = tid; idx < (int)MM; idx += nthr) sm[(idx / M) * ld + idx % M] = Akk[idx];
      __syncthreads();
      if (tid == 0) {
        const double piv = sm[0];
        const bool bad = !(fabs(piv) > 0.0) || !isfinite(piv);
        if (bad && blockIdx.x == 0) taps_flag(status, TAPS_DEV_SINGULAR);
        invd[0] = bad ? 1.0 : taps_rcp(piv);
      }
      __syncthreads();
      for (int p = 0; p < M - 1; ++p) {
        const double inv = invd[p];
        // warp 0 finishes row p+1 and the next pivot's reciprocal (the chain) alone;
        // warps 1 .. update the other rows four at a time (independent loads and FMAs
        // in flight)
        if (warp == 0) {
          const int r = p + 1;
          const double l = sm[r * ld + p] * inv;
          for (int c = p + 1 + lane; c < M; c += 32) sm[r * ld + c] = fma(-l, sm[p * ld + c], sm[r * ld + c]);
          __syncwarp();
          if (lane == 0) {
            sm[r * ld + p] = l;   // unit lower factor
            const double piv = sm[r * ld + r];
            const bool bad = !(fabs(piv) > 0.0) || !isfinite(piv);
            if (bad && blockIdx.x == 0) taps_flag(status, TAPS_DEV_SINGULAR);
            invd[r] = bad ? 1.0 : taps_rcp(piv);
          }
        } else {
          const int nwo = nwarps - 1;   // the other rows over warps 1 ..
          for (int rb = p + 1 + warp; rb < M; rb += 4 * nwo) {
            double l[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = rb + u * nwo;
              l[u] = r < M ? sm[r * ld + p] * inv : 0.0;
            }
            for (int c = p + 1 + lane; c < M; c += 32) {
              const double pc = sm[p * ld + c];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                const int r = rb + u * nwo;
                if (r < M) sm[r * ld + c] = fma(-l[u], pc, sm[r * ld + c]);
              }
            }
            __syncwarp();
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int r = rb + u * nwo;
              if (r < M && lane == 0) sm[r * ld + p] = l[u];
            }
          }
        }
        __syncthreads();
      }
      // ---- W(k, k+jj) = LU^{-1} A(k, k+jj), z_k = LU^{-1} F_k : one warp per column
      for (int task = blockIdx.x * nwarps + warp; task < ntask; task += (int)nblk * nwarps) {
        double* col;
        int cstride;
        if (task < nj * M) {
          int jj = task / M + 1, cc = task % M;
          col = BLK(k, k + jj) + cc;
          cstride = M;
        } else {
          col = F + (size_t)k * M;
          cstride = 1;
        }
        double v[4];
        // only the slots that hold rows issue FP64 work (a warp-wide FP64 instruction
        // holds the sub-partition's pipe however few lanes are active)
        const int nsl = (M + 31) >> 5;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          int r = lane + 32 * s;
          v[s] = (s < nsl && r < M) ? col[(size_t)r * cstride] : 0.0;
        }
        // forward: unit lower L
        for (int c = 0; c < M; ++c) {
          double yc = __shfl_sync(0xffffffffu, slot_get(v, c >> 5), c & 31);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            if (s >= nsl) break;
            int r = lane + 32 * s;
            const double a = (r > c && r < M) ? sm[r * ld + c] : 0.0;
            v[s] = fma(-a, yc, v[s]);
          }
        }
        // backward: upper U, with the kept reciprocals of its diagonal
        for (int c = M - 1; c >= 0; --c) {
          int sc = c >> 5;
          double own = slot_get(v, sc);
          if (lane == (c & 31)) {
            own *= invd[c];
            slot_set(v, sc, own);
          }
          double yc = __shfl_sync(0xffffffffu, own, c & 31);
#pragma unroll
          for (int s = 0; s < 4; ++s) {
            if (s >= nsl) break;
            int r = lane + 32 * s;
            const double a = (r < c) ? sm[r * ld + c] : 0.0;
            v[s] = fma(-a, yc, v[s]);
          }
        }
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          int r = lane + 32 * s;
          if (r < M) col[(size_t)r * cstride] = v[s];
        }
      }
    }
    grid_barrier(bar, status, nblk);

    // ---- Schur updates of the trailing window
    const long long nupd = (long long)nj * nj * MM;
    const long long total = nupd + (long long)nj * M;
    for (long long o = gtid; o < total; o += gthreads) {
      if (o < nupd) {
        int pair = (int)(o / MM);
        int rem = (int)(o % MM);
        int ii = pair / nj + 1, jj = pair % nj + 1;
        int m = rem / M, n = rem % M;
        const double* L = BLK(k + ii, k) + (size_t)m * M;
        const double* W = BLK(k, k + jj) + n;
        double s = 0.0;
        for (int l = 0; l < M; ++l) s = fma(L[l], W[(size_t)l * M], s);
        BLK(k + ii, k + jj)[(size_t)m * M + n] -= s;
      } else {
        int o2 = (int)(o - nupd);
        int ii = o2 / M + 1, m = o2 % M;
        const double* L = BLK(k + ii, k) + (size_t)m * M;
        const double* z = F + (size_t)k * M;
        double s = 0.0;
        for (int l = 0; l < M; ++l) s = fma(L[l], z[l], s);
        F[(size_t)(k + ii) * M + m] -= s;
      }
    }
    grid_barrier(bar, status, nblk);
  }
#undef BLK
}

// Back substitution x_k = z_k - sum_j W_kj x_j (k = nf-1 .. 0), written into the
// column-major factor U_d.  One CTA; each output is split over 8 partial dots.
__global__ void __launch_bounds__(256) block_backsub_kernel(const double* __restrict__ blocks,
                                                            const double* __restrict__ F, int nf,
                                                            int hb, int M, double* __restrict__ X,
                                                            int* status) {
  extern __shared__ __align__(16) double xs[];  // [(hb+1)][M] ring + [8][M] partials
  const int nb = 2 * hb + 1;
  const size_t MM = (size_t)M * M;
  double* part = xs + (size_t)(hb + 1) * M;
  const int tid = threadIdx.x;
  const int nparts = 8;
  for (int k = nf - 1; k >= 0; --k) {
    const int nj = min(hb, nf - 1 - k);
    const int work = nj * M;  // dot length per output
    for (int idx = tid; idx < nparts * M; idx += blockDim.x) {
      int m = idx % M, pp = idx / M;
      double s = 0.0;
      for (int w = pp; w < work; w += nparts) {
        int jj = w / M + 1, n = w % M;
        const double* W = blocks + ((size_t)k * nb + (jj + hb)) * MM;
        s += W[(size_t)m * M + n] * xs[((k + jj) % (hb + 1)) * M + n];
      }
      part[pp * M + m] = s;
    }
    __syncthreads();
    for (int m = tid; m < M; m += blockDim.x) {
      double s = F[(size_t)k * M + m];
      for (int pp = 0; pp < nparts; ++pp) s -= part[pp * M + m];
      if (!isfinite(s)) taps_flag(status, TAPS_DEV_NONFINITE);
      xs[(k % (hb + 1)) * M + m] = s;
      X[(size_t)m * nf + k] = s;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------------
// Column normalisation (unit 2-norm, largest-magnitude entry positive) and the
// squared change / norm of every column against the pre-solve copy.
// ---------------------------------------------------------------------------------
__global__ void normalize_change_kernel(double* U, const double* Uold, int nf, int M, int normalize,
                                        double* out, int* status) {
  taps_pdl_wait();
  __shared__ double red[32];
  __shared__ double redv[32];
  __shared__ int redi[32];
  int m = blockIdx.x;
  double* col = U + (size_t)m * nf;
  const double* old = Uold + (size_t)m * nf;
  double s2 = 0.0, best = -1.0;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    double v = col[i];
    s2 += v * v;
    double a = fabs(v);
    if (a > best) { best = a; bi = i; }
  }
  s2 = block_sum(s2, red);
  // argmax with ties to the smallest index
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { redv[w] = best; redi[w] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int nw = (blockDim.x + 31) >> 5;
    for (int j = 1; j < nw; ++j)
      if (redv[j] > redv[0] || (redv[j] == redv[0] && redi[j] < redi[0])) { redv[0] = redv[j]; redi[0] = redi[j]; }
  }
  __syncthreads();
  int imax = redi[0];
  double nrm = sqrt(s2);
  if (!isfinite(nrm)) taps_flag(status, TAPS_DEV_NONFINITE);
  if (normalize && nrm > 0.0) {
    double sgn = (col[imax] >= 0.0) ? 1.0 : -1.0;
    double den = sgn * nrm;
    __syncthreads();
    for (int i = threadIdx.x; i < nf; i += blockDim.x) col[i] = col[i] / den;
    __syncthreads();
  }
  double dif = 0.0, n2 = 0.0;
  for (int i = threadIdx.x; i < nf; i += blockDim.x) {
    double v = col[i];
    double dv = v - old[i];
    dif += dv * dv;
    n2 += v * v;
  }
  dif = block_sum(dif, red);
  n2 = block_sum(n2, red);
  if (threadIdx.x == 0) {
    out[2 * m] = dif;
    out[2 * m + 1] = n2;
  }
}

// The same for columns of at most NC_PER * 256 entries, with the column and its old
// values held in registers: one load of each, the sum of squares and the signed
// largest entry in one pass of reductions, the scaled column written once, and the
// change sums in a second pass.  Each sum follows the block_sum tree (per-thread order,
// xor butterfly in the warp, then the butterfly over the warps' sums in warp 0), so the
// results equal normalize_change_kernel's bit for bit.  The largest magnitude is found
// on the bit patterns of |v| (non-negative doubles order like their bits), the block
// totals and the square root in warp 0 only: every warp-wide FP64 instruction holds the
// pipe of its SM sub-partition for ~64 cycles on this GPU.
#define NC_PER 4
__global__ void __launch_bounds__(256) normalize_change_reg_kernel(double* U, const double* Uold, int nf, int M,
                                                                   int normalize, double* out, int* status) {
  __shared__ double rs[8], rsv[8], rd[8], rn[8];
  __shared__ long long rk[8];
  __shared__ int ri[8];
  __shared__ double den_s;
  taps_pdl_wait();
  const int m = blockIdx.x, lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  double* col = U + (size_t)m * nf;
  const double* old = Uold + (size_t)m * nf;
  double v[NC_PER], o[NC_PER];
#pragma unroll
  for (int k = 0; k < NC_PER; ++k) {
    const int i = threadIdx.x + k * 256;
    v[k] = i < nf ? col[i] : 0.0;
    o[k] = i < nf ? old[i] : 0.0;
  }
  double s2 = 0.0, bv = 0.0;
  long long best = -1;   // bits of |v|; -1 below every entry
  int bi = 0x7fffffff;
#pragma unroll
  for (int k = 0; k < NC_PER; ++k) {
    const int i = threadIdx.x + k * 256;
    if (i < nf) {
      s2 += v[k] * v[k];
      const long long a = __double_as_longlong(fabs(v[k]));
      if (a > best) { best = a; bi = i; bv = v[k]; }
    }
  }
  s2 = warp_sum(s2);
  // largest magnitude with ties to the smallest index, carrying its signed value
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    const long long ob = __shfl_xor_sync(0xffffffffu, best, o2);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o2);
    const double ov = __shfl_xor_sync(0xffffffffu, bv, o2);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; bv = ov; }
  }
  if (lane == 0) { rs[w] = s2; rk[w] = best; ri[w] = bi; rsv[w] = bv; }
  __syncthreads();
  const int nw = 8;
  if (w == 0) {
    const double tot = warp_sum(lane < nw ? rs[lane] : 0.0);
    if (lane == 0) {
      long long gb = rk[0];
      int gi = ri[0];
      double gv = rsv[0];
      for (int j = 1; j < nw; ++j)
        if (rk[j] > gb || (rk[j] == gb && ri[j] < gi)) { gb = rk[j]; gi = ri[j]; gv = rsv[j]; }
      const double nrm = sqrt(tot);
      if (!isfinite(nrm)) taps_flag(status, TAPS_DEV_NONFINITE);
      den_s = (normalize && nrm > 0.0) ? (gv >= 0.0 ? 1.0 : -1.0) * nrm : 0.0;
    }
  }
  __syncthreads();
  const double den = den_s;
  if (den != 0.0) {
#pragma unroll
    for (int k = 0; k < NC_PER; ++k) {
      const int i = threadIdx.x + k * 256;
      if (i < nf) {
        v[k] = v[k] / den;
        col[i] = v[k];
      }
    }
  }
  double dif = 0.0, n2 = 0.0;
#pragma unroll
  for (int k = 0; k < NC_PER; ++k) {
    const int i = threadIdx.x + k * 256;
    if (i < nf) {
      const double dv = v[k] - o[k];
      dif += dv * dv;
      n2 += v[k] * v[k];
    }
  }
  dif = warp_sum(dif);
  n2 = warp_sum(n2);
  if (lane == 0) { rd[w] = dif; rn[w] = n2; }
  __syncthreads();
  if (w == 0) {
    dif = warp_sum(lane < nw ? rd[lane] : 0.0);
    n2 = warp_sum(lane < nw ? rn[lane] : 0.0);
    if (lane == 0) {
      out[2 * m] = dif;
      out[2 * m + 1] = n2;
    }
  }
}

// ---------------------------------------------------------------------------------
// Reduced solve of dim d with the coefficients already in P->d_C / P->d_c.
// ---------------------------------------------------------------------------------
// Tile-shape tuner of the block elimination: the number of co-resident CTAs trades
// parallel work per block row against the cost of the three grid barriers per row.
// On first use for a (n, M) pair, outside any graph capture, each candidate runs the
// elimination on the current block band (re-assembled before every trial, so every
// trial computes the same thing) and the fastest is cached for the problem.
static int lu_grid_default(const taps_problem* P, int hb, int M) {
  int want = (int)std::min<long long>((long long)hb * hb * M * M / 256 + 1, P->num_sms);
  int want_a = (hb * M + 1 + 7) / 8;
  return std::min(std::max(1, std::max(want, want_a)), P->coop_blocks);
}

int taps_lu_grid(taps_problem* P, int d, taps_factors* U, int nf, int M) {
  const int hb = P->dims[d]->hb;
  for (int k = 0; k < P->n_lu_tuned; ++k)
    if (P->lu_tuned[k][0] == nf && P->lu_tuned[k][1] == M) return P->lu_tuned[k][2];
  int fallback = lu_grid_default(P, hb, M);
  if (P->prof->capturing || P->n_lu_tuned >= 16 || getenv("TAPS_NO_TUNE")) return fallback;
  const int cands[] = {8, 16, 32, 64, 96, 152};
  cudaStream_t s = P->stream;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return fallback;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return fallback; }
  // keep the assembled band: trials work on a copy
  const size_t band = sizeof(double) * ((size_t)nf * P->dims[d]->nb * M * M);
  const size_t rhs = sizeof(double) * (size_t)nf * M;
  double* keep = nullptr;
  if (taps_alloc((void**)&keep, band + rhs + sizeof(double)) != TAPS_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return fallback; }
  cudaMemcpyAsync(keep, P->d_blocks, band, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync((char*)keep + band, P->d_F, rhs, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync((char*)keep + band + rhs, P->d_status, sizeof(int), cudaMemcpyDeviceToDevice, s);
  int best = fallback;
  float best_ms = 1e30f;
  size_t smem = sizeof(double) * (size_t)M * (M + 1);
  int hbv = hb, nfv = nf, Mv = M;
  for (int c : cands) {
    int g = std::min(c, P->coop_blocks);
    cudaMemcpyAsync(P->d_blocks, keep, band, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(P->d_F, (char*)keep + band, rhs, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(P->d_bar, 0, 2 * sizeof(unsigned), s);
    double* blocks = P->d_blocks;
    double* Fp = P->d_F;
    double* lu = P->d_lu;
    int* st = P->d_status;
    unsigned* bar = P->d_bar;
    void* args[] = {&blocks, &Fp, &lu, &nfv, &hbv, &Mv, &st, &bar};
    cudaEventRecord(e0, s);
    if (cudaLaunchCooperativeKernel((const void*)block_lu_kernel, dim3(g), dim3(256), args, smem, s) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaEventRecord(e1, s);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = g; }
  }
  // restore the assembled band and the status word for the real elimination
  cudaMemcpyAsync(P->d_blocks, keep, band, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(P->d_F, (char*)keep + band, rhs, cudaMemcpyDeviceToDevice, s);
  cudaMemcpyAsync(P->d_status, (char*)keep + band + rhs, sizeof(int), cudaMemcpyDeviceToDevice, s);
  cudaStreamSynchronize(s);
  cudaFree(keep);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  P->lu_tuned[P->n_lu_tuned][0] = nf;
  P->lu_tuned[P->n_lu_tuned][1] = M;
  P->lu_tuned[P->n_lu_tuned][2] = best;
  P->n_lu_tuned++;
  (void)U;
  return best;
}

// 1 if some dim of the sweep would use block elimination with an untuned (n, M).
int taps_lu_needs_tuning(const taps_problem* P, int solver, int M) {
  if (getenv("TAPS_NO_TUNE")) return 0;
  for (int d = 0; d < P->D; ++d) {
    int sa, sb;
    (void)sa;
    (void)sb;
    if (taps_dim_route(P, d, solver, M) != TAPS_ROUTE_LU) continue;
    bool found = false;
    for (int k = 0; k < P->n_lu_tuned; ++k)
      if (P->lu_tuned[k][0] == P->dims[d]->nf && P->lu_tuned[k][1] == M) found = true;
    if (!found && P->n_lu_tuned < 16) return 1;
  }
  return 0;
}

static int reduced_solve_block_lu(taps_problem* P, taps_factors* U, int d) {
  const taps_dim* dm = P->dims[d];
  int M = U->M, nf = dm->nf, hb = dm->hb, nb = dm->nb, nops = P->tt.nops[d];
  cudaStream_t s = P->stream;
  long long nblk = (long long)nf * nb * M * M + (long long)nf * M;
  int tk = prof_begin(P, TAPS_PROF_BLOCK_ASSEMBLE);
  block_assemble_kernel<<<(unsigned)((nblk + 255) / 256), 256, 0, s>>>(
      P->d_opband[d], nops, nf, nb, M, P->d_C, P->d_q[d], P->d_c, P->Rf, P->d_blocks, P->d_F);
  prof_end(P, TAPS_PROF_BLOCK_ASSEMBLE, tk, 2.0 * nops * (double)nf * nb * M * M + 2.0 * P->Rf * nf * M,
           8.0 * ((double)nf * nb * M * M + (double)nf * M + (double)nops * nf * nb + (double)P->Rf * nf));
  TAPS_CUDA(cudaGetLastError());
  // algorithmic flops of the elimination and of the back substitution
  double lu_flops = 0.0, bs_flops = 0.0;
  const double Md = M;
  for (int k = 0; k < nf; ++k) {
    int nj = std::min(hb, nf - 1 - k);
    lu_flops += (2.0 / 3.0) * Md * Md * Md + (nj * Md + 1) * 2.0 * Md * Md +
                nj * (double)nj * 2.0 * Md * Md * Md + nj * 2.0 * Md * Md;
    bs_flops += nj * 2.0 * Md * Md;
  }
  const double band_bytes = 8.0 * (double)nf * nb * M * M;
  // cooperative elimination; the CTA count comes from the tuner (first use per (n, M))
  size_t smem = sizeof(double) * (size_t)M * (M + 1);
  int grid = taps_lu_grid(P, d, U, nf, M);
  TAPS_CUDA(cudaMemsetAsync(P->d_bar, 0, 2 * sizeof(unsigned), s));
  double* blocks = P->d_blocks;
  double* Fp = P->d_F;
  double* lu = P->d_lu;
  int* st = P->d_status;
  unsigned* bar = P->d_bar;
  void* args[] = {&blocks, &Fp, &lu, &nf, &hb, &M, &st, &bar};
  tk = prof_begin(P, TAPS_PROF_BLOCK_LU);
  TAPS_CUDA(cudaLaunchCooperativeKernel((const void*)block_lu_kernel, dim3(grid), dim3(256), args,
                                        smem, s));
  prof_end(P, TAPS_PROF_BLOCK_LU, tk, lu_flops, 2.0 * band_bytes + 16.0 * nf * M);
  size_t smem_b = sizeof(double) * ((size_t)(hb + 1) * M + 8 * (size_t)M);
  tk = prof_begin(P, TAPS_PROF_BACKSUB);
  block_backsub_kernel<<<1, 256, smem_b, s>>>(P->d_blocks, P->d_F, nf, hb, M, U->d_U[d],
                                              P->d_status);
  prof_end(P, TAPS_PROF_BACKSUB, tk, bs_flops, 8.0 * (double)nf * hb * M * M + 16.0 * nf * M);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

static int residual_setup(int maxsm);

// Largest dynamic shared memory a launch of `fn` may ask for: the opt-in limit less
// the kernel's static shared memory.
int taps_allow_dyn_smem(const void* fn, int maxsm) {
  cudaFuncAttributes fa;
  TAPS_CUDA(cudaFuncGetAttributes(&fa, fn));
  TAPS_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 maxsm - (int)fa.sharedSizeBytes));
  return TAPS_OK;
}

// Shared-memory opt-in of the kernels whose footprint grows with M, and the number
// of CTAs a cooperative block-LU launch may use (co-residency at the largest M).
int taps_sweep_setup(int dev, int num_sms, int* coop_blocks) {
  int maxsm = 0;
  TAPS_CUDA(cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  TAPS_TRY(taps_allow_dyn_smem((const void*)block_lu_kernel, maxsm));
  TAPS_TRY(taps_allow_dyn_smem((const void*)gram_partial_kernel<double, false>, maxsm));
  TAPS_TRY(taps_allow_dyn_smem((const void*)gram_partial_kernel<float, false>, maxsm));
  TAPS_TRY(taps_allow_dyn_smem((const void*)gram_partial_kernel<float, true>, maxsm));
  TAPS_TRY(taps_allow_dyn_smem((const void*)gram_partial_all_kernel, maxsm));
  TAPS_TRY(residual_setup(maxsm));
  TAPS_TRY(taps_md_setup(maxsm));
  TAPS_TRY(taps_gram_tc_setup(maxsm));
  int bps = 0;
  size_t smem_max = sizeof(double) * TAPS_MAX_M * (TAPS_MAX_M + 1);
  TAPS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, block_lu_kernel, 256, smem_max));
  *coop_blocks = std::max(bps, 1) * num_sms;
  return TAPS_OK;
}

static int coefficients(taps_problem* P, int d, int M) {
  int tk = prof_begin(P, TAPS_PROF_COEFF);
  if (P->tt.cs > TAPS_NUM_OPS)
    TAPS_CUDA(taps_launch_pdl(coeff_slots_kernel, dim3((std::max(M * M, P->Rf * M) + 127) / 128), dim3(128), 0, P->stream, P->tt,
                              gram_ptrs(P), d, M, P->d_C, P->d_c));
  else
    TAPS_CUDA(taps_launch_pdl(coeff_kernel, dim3((std::max(M * M, P->Rf * M) + 127) / 128), dim3(128), 0, P->stream, P->tt,
                              gram_ptrs(P), d, M, P->d_C, P->d_c));
  prof_end(P, TAPS_PROF_COEFF, tk, (double)P->R * M * M * P->D + (double)P->Rf * M * P->D,
           8.0 * ((double)P->R * M * M * P->D));
  TAPS_CUDA(cudaGetLastError());
  P->c0_valid = (d == 0);
  P->c0_M = M;
  return TAPS_OK;
}

int taps_coefficients(taps_problem* P, int d, int M) { return coefficients(P, d, M); }

// Kernels of one sweep (no host synchronisation: capturable in a CUDA graph).  The
// per-column change / norm partials and the status word are copied to pinned host
// memory at the end; taps_sweep_finish reads them after the stream has drained.
int taps_sweep_enqueue(taps_problem* P, taps_factors* U, int precision, int solver, int normalize,
                       int host_copies) {
  int M = U->M;
  if (M < 1 || M > P->ws_M) return TAPS_ERR_INVALID_ARG;
  cudaStream_t s = P->stream;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    // the coefficients of the later dims come with the previous dim's Gram refresh, and
    // dim 0's with the last dim's refresh of the previous sweep (or of taps_refresh_grams)
    if (d == 0) {
      if (P->c0_valid && P->c0_M == M && !P->c0_forbid) P->c0_skipped = 1;
      else TAPS_TRY(coefficients(P, 0, M));
    }
    const int route = taps_dim_route(P, d, solver, M);
    if (route == TAPS_ROUTE_FD) {
      TAPS_TRY(taps_fd_solve(P, U, d, precision));   // keeps the old factor in d_Uold
    } else if (route == TAPS_ROUTE_MD) {
      TAPS_TRY(taps_md_solve(P, U, d));              // keeps the old factor in d_Uold
    } else if (route == TAPS_ROUTE_FDW) {
      TAPS_TRY(taps_fdw_solve(P, U, d));             // keeps the old factor in d_Uold
    } else {
      TAPS_CUDA(cudaMemcpyAsync(P->d_Uold, U->d_U[d], sizeof(double) * dm->nf * M,
                                cudaMemcpyDeviceToDevice, s));
      TAPS_TRY(reduced_solve_block_lu(P, U, d));
    }
    int norm_d = (normalize && d < P->D - 1) ? 1 : 0;
    int tk = prof_begin(P, TAPS_PROF_NORMALIZE);
    TAPS_CUDA(taps_launch_pdl(dm->nf <= NC_PER * 256 ? normalize_change_reg_kernel : normalize_change_kernel,
                              dim3(M), dim3(256), 0, s, U->d_U[d], (const double*)P->d_Uold, dm->nf, M, norm_d,
                              P->d_scal + (size_t)d * 2 * M, P->d_status));
    prof_end(P, TAPS_PROF_NORMALIZE, tk, 7.0 * dm->nf * M, 8.0 * 3.0 * dm->nf * M);
    TAPS_CUDA(cudaGetLastError());
    TAPS_TRY(taps_refresh_gram_dim(P, U, d, precision, d + 1 < P->D ? d + 1 : 0));
  }
  if (!host_copies) return TAPS_OK;
  return taps_results_to_host(P, 2 * M * P->D, 0);
}

// Reads the device status and the change partials copied by taps_sweep_enqueue (the
// caller has synchronised the stream).
int taps_sweep_finish(taps_problem* P, taps_factors* U, double* change_out) {
  int M = U->M;
  if (*P->h_status != TAPS_DEV_OK) {
    int dev = *P->h_status;
    *P->h_status = TAPS_DEV_OK;
    TAPS_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), P->stream));
    TAPS_CUDA(cudaStreamSynchronize(P->stream));
    return taps_status_from_device(dev);
  }
  prof_drain(P);
  double change = 0.0;
  for (int d = 0; d < P->D; ++d) {
    double dif = 0.0, n2 = 0.0;
    for (int m = 0; m < M; ++m) {
      dif += P->h_scal[(size_t)d * 2 * M + 2 * m];
      n2 += P->h_scal[(size_t)d * 2 * M + 2 * m + 1];
    }
    double ch = n2 > 0.0 ? sqrt(dif / n2) : INFINITY;
    change = std::max(change, ch);
  }
  if (!std::isfinite(change)) return TAPS_ERR_NONFINITE;
  if (change_out) *change_out = change;
  return TAPS_OK;
}

int taps_sweep_impl(taps_problem* P, taps_factors* U, int precision, int solver, int normalize,
                    double* change_out) {
  int M = U->M;
  if (M < 1) return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_ws_ensure(P, M));
  TAPS_TRY(taps_fd_prepare_all(P, solver, M));
  TAPS_TRY(taps_sweep_enqueue(P, U, precision, solver, normalize));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return taps_sweep_finish(P, U, change_out);
}

// ---------------------------------------------------------------------------------
// Residuals
// ---------------------------------------------------------------------------------
// Y_o = Op_o U for every distinct op of dim d; Y layout [nops][nf][M] (row-major).
__global__ void spmm_kernel(const double* __restrict__ U, int nf, int M, int hb,
                            const double* __restrict__ opband, int nops, double* __restrict__ Y) {
  long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long tot = (long long)nops * nf * M;
  if (idx >= tot) return;
  int m = idx % M;
  int i = (idx / M) % nf;
  int o = idx / ((long long)M * nf);
  int nb = 2 * hb + 1;
  const double* brow = opband + ((size_t)o * nf + i) * nb;
  double acc = 0.0;
  for (int k = 0; k < nb; ++k) {
    int j = i + k - hb;
    if (j >= 0 && j < nf) acc += brow[k] * U[(size_t)m * nf + j];
  }
  Y[idx] = acc;
}

// Residual of every dim's reduced system at the current factors (Eq. 42):
// r_d[i][m] = sum_o (Op_o U_d)[i][:] . C_{d,o}[m][:] - sum_r q_{d,r}[i] c_{d,r}[m].
// One launch for all dims: CTA b belongs to the dim whose range [cta0[d], cta0[d+1])
// holds b and covers RR rows of it.  The CTA stages the factor rows with their band
// halo and Y_o = Op_o U on those rows in shared memory, then writes its partial sums
// of ||r||^2 and ||F||^2 (summed per dim in a fixed order on the host).
#define RR 8
struct ResDims {
  const double* U[TAPS_MAX_DIMS];
  const double* band[TAPS_MAX_DIMS];   // [nops][nf][nb]
  const double* q[TAPS_MAX_DIMS];      // [Rf][nf]
  int nf[TAPS_MAX_DIMS], hb[TAPS_MAX_DIMS], nops[TAPS_MAX_DIMS];
  int cta0[TAPS_MAX_DIMS + 1];
  int D;
  int cs;   // slot stride of Call
};

__global__ void __launch_bounds__(256) als_residual_all_kernel(ResDims rd, int M, int Rf,
                                                               const double* __restrict__ Call,
                                                               const double* __restrict__ call,
                                                               double* __restrict__ partial) {
  extern __shared__ __align__(16) double rsm[];
  __shared__ double red[32];
  const int b = blockIdx.x;
  taps_pdl_wait();
  int d = 0;
  while (d + 1 < rd.D && b >= rd.cta0[d + 1]) ++d;
  const int r0 = (b - rd.cta0[d]) * RR;
  const int nf = rd.nf[d], hb = rd.hb[d], nops = rd.nops[d], nb = 2 * hb + 1;
  const int rows_h = RR + 2 * hb;
  double* Us = rsm;                 // [rows_h][M]
  double* Ys = Us + rows_h * M;     // [nops][RR][M]
  const double* U = rd.U[d];
  for (int idx = threadIdx.x; idx < rows_h * M; idx += blockDim.x) {
    const int m = idx / rows_h, rr = idx % rows_h;
    const int gi = r0 - hb + rr;
    Us[rr * M + m] = (gi >= 0 && gi < nf) ? U[(size_t)m * nf + gi] : 0.0;
  }
  __syncthreads();
  for (int o = 0; o < nops; ++o) {
    const double* band = rd.band[d] + (size_t)o * nf * nb;
    for (int idx = threadIdx.x; idx < RR * M; idx += blockDim.x) {
      const int i = idx / M, n = idx % M;
      const int gi = r0 + i;
      double acc = 0.0;
      if (gi < nf) {
        const double* brow = band + (size_t)gi * nb;
        for (int k = 0; k < nb; ++k) acc += brow[k] * Us[(i + k) * M + n];
      }
      Ys[(o * RR + i) * M + n] = acc;
    }
  }
  __syncthreads();
  const double* C = Call + (size_t)d * rd.cs * M * M;
  const double* c = call + (size_t)d * Rf * M;
  const double* q = rd.q[d];
  double r2 = 0.0, f2 = 0.0;
  for (int idx = threadIdx.x; idx < RR * M; idx += blockDim.x) {
    const int i = idx / M, m = idx % M;
    const int gi = r0 + i;
    if (gi < nf) {
      double f = 0.0;
      for (int r = 0; r < Rf; ++r) f += q[(size_t)r * nf + gi] * c[(size_t)r * M + m];
      double a = 0.0;
      for (int o = 0; o < nops; ++o) {
        const double* y = Ys + (o * RR + i) * M;
        const double* cc = C + ((size_t)o * M + m) * M;
        for (int n = 0; n < M; ++n) a += y[n] * cc[n];
      }
      const double rr = a - f;
      r2 += rr * rr;
      f2 += f * f;
    }
  }
  r2 = block_sum(r2, red);
  f2 = block_sum(f2, red);
  if (threadIdx.x == 0) {
    partial[2 * b] = r2;
    partial[2 * b + 1] = f2;
  }
}

static int residual_setup(int maxsm) {
  TAPS_TRY(taps_allow_dyn_smem((const void*)als_residual_all_kernel, maxsm));
  return TAPS_OK;
}

// Per-dim Gram of the columns [Y_0 | Y_1 | ... | q_0 .. q_{Rf-1}] (NC = nops*M + Rf).
// CTA a forms row a: its threads split the columns b (BG_COLS at a time) and the
// rows i (BG_SPLIT ways, so that each thread's chain of products is short and its
// loads overlap); the row splits are summed in a fixed order through shared memory.
#define BG_COLS 64
#define BG_SPLIT 4
__device__ __forceinline__ double big_gram_col(const double* Y, const double* q, int nops, int nf, int M,
                                               int a, int i) {
  return (a < nops * M) ? Y[((size_t)(a / M) * nf + i) * M + (a % M)] : q[(size_t)(a - nops * M) * nf + i];
}

struct BigGramPtrs {
  const double* G[TAPS_MAX_DIMS];
  int NC[TAPS_MAX_DIMS];
};

// Every dim of the full residual in one launch each: the banded products Y_o = Op_o U
// of all dims (thread per output, as spmm_kernel) and the big Grams of all dims (CTA per
// pair of rows of dim d's Gram of the columns [Y_0 .. Y_{nops-1} | Q]: per entry
// BG_SPLIT row ranges, each a sequential sum taking its operands eight rows at a time so
// that their loads are in flight together, then the ranges' sums added pairwise).
struct ResAll {
  const double* U[TAPS_MAX_DIMS];
  const double* band[TAPS_MAX_DIMS];
  const double* q[TAPS_MAX_DIMS];
  double* G[TAPS_MAX_DIMS];
  long long yoff[TAPS_MAX_DIMS + 1];   // prefix of nops_d nf_d M (outputs of the banded products)
  int aoff[TAPS_MAX_DIMS + 1];         // prefix of NC_d (rows of the big Grams)
  int nf[TAPS_MAX_DIMS], hb[TAPS_MAX_DIMS], nops[TAPS_MAX_DIMS];
  int D;
};

__global__ void spmm_all_kernel(ResAll ra, int M, double* __restrict__ Yall) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= ra.yoff[ra.D]) return;
  int d = 0;
  while (d + 1 < ra.D && idx >= ra.yoff[d + 1]) ++d;
  const long long loc = idx - ra.yoff[d];
  const int nf = ra.nf[d], hb = ra.hb[d], nb = 2 * hb + 1;
  const int m = loc % M;
  const int i = (loc / M) % nf;
  const int o = loc / ((long long)M * nf);
  const double* brow = ra.band[d] + ((size_t)o * nf + i) * nb;
  const double* U = ra.U[d];
  double acc = 0.0;
  for (int k = 0; k < nb; ++k) {
    int j = i + k - hb;
    if (j >= 0 && j < nf) acc += brow[k] * U[(size_t)m * nf + j];
  }
  Yall[idx] = acc;
}

__global__ void __launch_bounds__(BG_COLS * BG_SPLIT) big_gram_all_kernel(ResAll ra, int M, int Rf,
                                                                           const double* __restrict__ Yall,
                                                                           int stage) {
  extern __shared__ double ysm[];   // [2][nf]: the columns of the CTA's two rows (stage)
  __shared__ double part[BG_SPLIT][BG_COLS];
  int d = 0;
  while (d + 1 < ra.D && (int)blockIdx.x >= ra.aoff[d + 1]) ++d;
  const int nops = ra.nops[d], nf = ra.nf[d];
  const int NC = nops * M + Rf;
  // the Gram is symmetric and a product does not depend on its operands' order, so
  // entry (a, b) is formed once for b >= a and written to both places; the CTA takes
  // rows pr and NC-1-pr (NC + 1 columns between them, the middle row alone)
  const int pr = blockIdx.x - ra.aoff[d];
  const int r0 = pr, r1 = NC - 1 - pr;
  const int len0 = NC - r0;
  const int nv = (r1 == r0) ? len0 : len0 + (NC - r1);
  const double* Y = Yall + ra.yoff[d];
  const double* q = ra.q[d];
  if (stage) {
    for (int i = threadIdx.x; i < nf; i += blockDim.x) {
      ysm[i] = big_gram_col(Y, q, nops, nf, M, r0, i);
      ysm[nf + i] = big_gram_col(Y, q, nops, nf, M, r1, i);
    }
    __syncthreads();
  }
  const int col = threadIdx.x % BG_COLS, sp = threadIdx.x / BG_COLS;
  const int i0 = (int)((long long)nf * sp / BG_SPLIT), i1 = (int)((long long)nf * (sp + 1) / BG_SPLIT);
  for (int v0 = 0; v0 < nv; v0 += BG_COLS) {
    const int v = v0 + col;
    int a = -1, b = 0;
    if (v < nv) {
      if (v < len0) { a = r0; b = r0 + v; }
      else { a = r1; b = r1 + (v - len0); }
    }
    const double* xs = ysm + (a == r0 ? 0 : nf);
    double acc = 0.0;
    if (a >= 0) {
      int i = i0;
      for (; i + 8 <= i1; i += 8) {
        double x[8], y[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          x[k] = stage ? xs[i + k] : big_gram_col(Y, q, nops, nf, M, a, i + k);
          y[k] = big_gram_col(Y, q, nops, nf, M, b, i + k);
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) acc += x[k] * y[k];
      }
      for (; i < i1; ++i)
        acc += (stage ? xs[i] : big_gram_col(Y, q, nops, nf, M, a, i)) * big_gram_col(Y, q, nops, nf, M, b, i);
    }
    part[sp][col] = acc;
    __syncthreads();
    if (sp == 0 && a >= 0) {
      const double g = (part[0][col] + part[1][col]) + (part[2][col] + part[3][col]);
      ra.G[d][(size_t)a * NC + b] = g;
      ra.G[d][(size_t)b * NC + a] = g;
    }
    __syncthreads();
  }
}

// Gram-identity combination: partial sums of ||F||^2, F^T A u and ||A u||^2.
__global__ void full_residual_combine_kernel(TermTable tt, BigGramPtrs bg, int M, double* partial) {
  __shared__ double red[32];
  const long long nAA = (long long)tt.R * M * tt.R * M;
  const long long nFA = (long long)tt.Rf * tt.R * M;
  const long long nFF = (long long)tt.Rf * tt.Rf;
  const long long tot = nAA + nFA + nFF;
  double sAA = 0.0, sFA = 0.0, sFF = 0.0;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < tot;
       idx += (long long)gridDim.x * blockDim.x) {
    if (idx < nAA) {
      int tm = idx / ((long long)tt.R * M), sn = idx % ((long long)tt.R * M);
      int t = tm / M, m = tm % M, t2 = sn / M, n = sn % M;
      double v = tt.alpha[t] * tt.alpha[t2];
      for (int d = 0; d < tt.D; ++d)
        v *= bg.G[d][(size_t)(tt.oi[t][d] * M + m) * bg.NC[d] + tt.oi[t2][d] * M + n];
      sAA += v;
    } else if (idx < nAA + nFA) {
      long long j = idx - nAA;
      int r = j / ((long long)tt.R * M), tm = j % ((long long)tt.R * M);
      int t = tm / M, m = tm % M;
      double v = tt.beta[r] * tt.alpha[t];
      for (int d = 0; d < tt.D; ++d) {
        int qa = tt.nops[d] * M + r;
        v *= bg.G[d][(size_t)qa * bg.NC[d] + tt.oi[t][d] * M + m];
      }
      sFA += v;
    } else {
      long long j = idx - nAA - nFA;
      int r = j / tt.Rf, r2 = j % tt.Rf;
      double v = tt.beta[r] * tt.beta[r2];
      for (int d = 0; d < tt.D; ++d) {
        int qa = tt.nops[d] * M + r, qb = tt.nops[d] * M + r2;
        v *= bg.G[d][(size_t)qa * bg.NC[d] + qb];
      }
      sFF += v;
    }
  }
  sAA = block_sum(sAA, red);
  sFA = block_sum(sFA, red);
  sFF = block_sum(sFF, red);
  if (threadIdx.x == 0) {
    partial[3 * blockIdx.x] = sFF;
    partial[3 * blockIdx.x + 1] = sFA;
    partial[3 * blockIdx.x + 2] = sAA;
  }
}

// Residual kernels (no host synchronisation); the partial sums land in pinned host
// memory (P->h_part) for taps_residual_finish.  Returns the number of partials.
int taps_residual_enqueue(taps_problem* P, const taps_factors* U, int kind, int grams_current,
                          int host_copies) {
  int M = U->M;
  if (M < 1 || M > P->ws_M) return TAPS_ERR_INVALID_ARG;
  cudaStream_t s = P->stream;
  if (kind == TAPS_RES_ALS) {
    // FP64 Grams of every dim at the current factors, the coefficients of every dim,
    // then every dim's residual in one launch.
    if (!grams_current) TAPS_TRY(taps_refresh_grams(P, U, TAPS_FP64));
    int tk = prof_begin(P, TAPS_PROF_COEFF);
    if (P->tt.cs > TAPS_NUM_OPS)
      TAPS_CUDA(taps_launch_pdl(coeff_all_slots_kernel, dim3((std::max(M * M, P->Rf * M) + 127) / 128, P->D), dim3(128), 0, s,
                                P->tt, gram_ptrs(P), M, P->d_Call, P->d_call));
    else
      TAPS_CUDA(taps_launch_pdl(coeff_all_kernel, dim3((std::max(M * M, P->Rf * M) + 127) / 128, P->D), dim3(128), 0, s, P->tt,
                                gram_ptrs(P), M, P->d_Call, P->d_call));
    prof_end(P, TAPS_PROF_COEFF, tk, (double)P->R * M * M * P->D * P->D,
             8.0 * ((double)P->R * M * M * P->D * P->D));
    TAPS_CUDA(cudaGetLastError());
    ResDims rd;
    memset(&rd, 0, sizeof(rd));
    rd.D = P->D;
    rd.cs = P->tt.cs;
    double fl = 0.0, by = 0.0;
    int rows_max = 0;
    for (int d = 0; d < P->D; ++d) {
      const taps_dim* dm = P->dims[d];
      rd.U[d] = U->d_U[d];
      rd.band[d] = P->d_opband[d];
      rd.q[d] = P->d_q[d];
      rd.nf[d] = dm->nf;
      rd.hb[d] = dm->hb;
      rd.nops[d] = P->tt.nops[d];
      rd.cta0[d + 1] = rd.cta0[d] + (dm->nf + RR - 1) / RR;
      rows_max = std::max(rows_max, RR + 2 * dm->hb + P->tt.nops[d] * RR);
      const double ny = (double)rd.nops[d] * dm->nf * M, nr = (double)dm->nf * M;
      fl += 2.0 * ny * dm->nb + 2.0 * rd.nops[d] * nr * M + 2.0 * P->Rf * nr;
      by += 8.0 * (nr + (double)rd.nops[d] * dm->nf * dm->nb + (double)P->Rf * dm->nf);
    }
    tk = prof_begin(P, TAPS_PROF_RESIDUAL);
    TAPS_CUDA(taps_launch_pdl(als_residual_all_kernel, dim3(rd.cta0[P->D]), dim3(256),
                              sizeof(double) * (size_t)rows_max * M, s, rd, M, P->Rf,
                              (const double*)P->d_Call, (const double*)P->d_call, P->d_partial));
    prof_end(P, TAPS_PROF_RESIDUAL, tk, fl, by);
    TAPS_CUDA(cudaGetLastError());
    if (!host_copies) return TAPS_OK;
    return taps_results_to_host(P, 0, taps_residual_npart(P, TAPS_RES_ALS));
  }
  if (kind != TAPS_RES_FULL) return TAPS_ERR_INVALID_ARG;
  BigGramPtrs bg;
  memset(&bg, 0, sizeof(bg));
  ResAll ra;
  memset(&ra, 0, sizeof(ra));
  ra.D = P->D;
  size_t goff = 0;
  double fl = 0.0, by = 0.0;
  for (int d = 0; d < P->D; ++d) {
    const taps_dim* dm = P->dims[d];
    int nops = P->tt.nops[d];
    int NC = nops * M + P->Rf;
    long long ny = (long long)nops * dm->nf * M;
    ra.U[d] = U->d_U[d];
    ra.band[d] = P->d_opband[d];
    ra.q[d] = P->d_q[d];
    ra.G[d] = P->d_bigG + goff;
    ra.nf[d] = dm->nf;
    ra.hb[d] = dm->hb;
    ra.nops[d] = nops;
    ra.yoff[d + 1] = ra.yoff[d] + ny;
    ra.aoff[d + 1] = ra.aoff[d] + (NC + 1) / 2;   // row pairs of the symmetric big Gram
    fl += 2.0 * ny * dm->nb + 2.0 * (double)NC * NC * dm->nf;
    by += 8.0 * 2.0 * ny;
    bg.G[d] = P->d_bigG + goff;
    bg.NC[d] = NC;
    goff += (size_t)NC * NC;
  }
  {
    int tk = prof_begin(P, TAPS_PROF_RESIDUAL);
    const long long ny = ra.yoff[P->D];
    spmm_all_kernel<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(ra, M, P->d_Yres);
    TAPS_CUDA(cudaGetLastError());
    // the two rows' columns in shared memory when they fit the default 48 KB
    const int stage = (size_t)2 * P->nf_max * sizeof(double) <= 48 * 1024 ? 1 : 0;
    big_gram_all_kernel<<<ra.aoff[P->D], BG_COLS * BG_SPLIT, stage ? 2 * P->nf_max * sizeof(double) : 0, s>>>(
        ra, M, P->Rf, (const double*)P->d_Yres, stage);
    TAPS_CUDA(cudaGetLastError());
    P->prof->launches[TAPS_PROF_RESIDUAL] += 1;
    prof_end(P, TAPS_PROF_RESIDUAL, tk, fl, by);
  }
  const int nblk = 64;
  int tk = prof_begin(P, TAPS_PROF_RESIDUAL);
  full_residual_combine_kernel<<<nblk, 256, 0, s>>>(P->tt, bg, M, P->d_partial);
  prof_end(P, TAPS_PROF_RESIDUAL, tk, (double)P->R * M * P->R * M * (P->D + 1), 8.0 * (double)goff);
  TAPS_CUDA(cudaGetLastError());
  if (!host_copies) return TAPS_OK;
  return taps_results_to_host(P, 0, taps_residual_npart(P, TAPS_RES_FULL));
}

// The change partials of a sweep (nscal), the partial sums of a residual (npart) and the
// status word into the pinned host buffers (device-accessible under unified addressing)
// by one kernel: it replaces device-to-host copies of a few hundred bytes each, whose
// latency (several microseconds per copy) sat on the critical path of every sweep.
__global__ void host_results_kernel(const double* __restrict__ scal, int nscal, const double* __restrict__ part,
                                    int npart, const int* __restrict__ status, double* h_scal, double* h_part,
                                    int* h_status) {
  taps_pdl_wait();
  for (int i = threadIdx.x; i < nscal; i += blockDim.x) h_scal[i] = scal[i];
  for (int i = threadIdx.x; i < npart; i += blockDim.x) h_part[i] = part[i];
  if (threadIdx.x == 0) *h_status = *status;
  __threadfence_system();
}

int taps_residual_npart(const taps_problem* P, int kind) {
  if (kind != TAPS_RES_ALS) return 3 * 64;
  int cta0[TAPS_MAX_DIMS + 1];
  taps_als_partial_ranges(P, cta0);
  return 2 * cta0[P->D];
}

int taps_results_to_host(taps_problem* P, int nscal, int npart) {
  int tk = prof_begin(P, TAPS_PROF_OTHER);
  TAPS_CUDA(taps_launch_pdl(host_results_kernel, dim3(1), dim3(256), 0, P->stream, (const double*)P->d_scal,
                            nscal, (const double*)P->d_partial, npart, (const int*)P->d_status, P->h_scal,
                            P->h_part, P->h_status));
  prof_end(P, TAPS_PROF_OTHER, tk, 0.0, 8.0 * ((double)nscal + npart));
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}

int taps_als_partial_ranges(const taps_problem* P, int* cta0) {
  cta0[0] = 0;
  for (int d = 0; d < P->D; ++d) cta0[d + 1] = cta0[d] + (P->dims[d]->nf + RR - 1) / RR;
  return TAPS_OK;
}

int taps_residual_finish(taps_problem* P, const taps_factors* U, int kind, double* rho_out) {
  (void)U;
  if (*P->h_status != TAPS_DEV_OK) {
    int dev = *P->h_status;
    *P->h_status = TAPS_DEV_OK;
    TAPS_CUDA(cudaMemsetAsync(P->d_status, 0, sizeof(int), P->stream));
    TAPS_CUDA(cudaStreamSynchronize(P->stream));
    return taps_status_from_device(dev);
  }
  prof_drain(P);
  if (kind == TAPS_RES_ALS) {
    double worst = 0.0;
    size_t off = 0;
    for (int d = 0; d < P->D; ++d) {
      int nblocks = (P->dims[d]->nf + RR - 1) / RR;
      double r2 = 0.0, f2 = 0.0;
      for (int b = 0; b < nblocks; ++b) {
        r2 += P->h_part[off + 2 * b];
        f2 += P->h_part[off + 2 * b + 1];
      }
      off += 2 * (size_t)nblocks;
      double v = f2 > 0.0 ? sqrt(r2 / f2) : INFINITY;
      worst = std::max(worst, v);
    }
    if (!std::isfinite(worst)) return TAPS_ERR_NONFINITE;
    *rho_out = worst;
    return TAPS_OK;
  }
  double FF = 0.0, FA = 0.0, AA = 0.0;
  for (int b = 0; b < 64; ++b) {
    FF += P->h_part[3 * b];
    FA += P->h_part[3 * b + 1];
    AA += P->h_part[3 * b + 2];
  }
  double r2 = FF - 2.0 * FA + AA;
  double rho = sqrt(std::max(r2, 0.0) / FF);
  if (!std::isfinite(rho)) return TAPS_ERR_NONFINITE;
  *rho_out = rho;
  return TAPS_OK;
}

int taps_residual_impl(taps_problem* P, const taps_factors* U, int kind, double* rho_out,
                       int grams_current) {
  int M = U->M;
  if (M < 1) return TAPS_ERR_INVALID_ARG;
  TAPS_TRY(taps_ws_ensure(P, M));
  TAPS_TRY(taps_residual_enqueue(P, U, kind, grams_current));
  TAPS_CUDA(cudaStreamSynchronize(P->stream));
  return taps_residual_finish(P, U, kind, rho_out);
}
