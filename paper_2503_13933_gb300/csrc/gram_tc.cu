// Gram refresh on the 5th-generation tensor cores: BF16 operands, FP32 accumulation.
//
// For one dim of one instance (an "item") the refresh computes, for every distinct
// operator o of the dim and every source term r (Eq. 34),
//     Gamma_o = U^T (Op_o U)   (M x M),      h_r = U^T q_r   (M),
// with U the n x M factor, Op_o banded (half-width hb) and q_r the source projection.
// The reduced-precision contract of TAPS_BF16 holds here: U, the bands and the source
// vectors are rounded to bfloat16; the banded product Y_o = Op_o U is formed on the
// CUDA cores in FP32 and split as Y = Y_hi + Y_lo with both parts bfloat16 (so Y keeps
// ~16 significant bits); the contractions over the nodes run as tcgen05.mma
// kind::f16 with BF16 A and B and FP32 accumulators in tensor memory:
//     Gamma_o += U^T Y_hi + U^T Y_lo,   h += U^T Q   (one MMA per 16 nodes each).
// A = U^T is the mode-by-node tile (128 MMA rows, the item's M modes used), B = Y^T
// (N = M rounded up to 16) and Q (N_h = R_f rounded up to 16), all K-major in the
// no-swizzle core-matrix layout (8 rows x 16 bytes).
//
// Work decomposition: an item's nodes are cut into chunks of ROWS; a task is a run of
// chunks of one item, accumulated in TMEM by one CTA.  An item of one task writes its
// Grams directly; an item of several tasks writes per-task partials and the last task
// to finish (ticket counter, no waiting) sums them in task order, so the result does
// not depend on scheduling.  Two launch modes:
//   queue  - persistent CTAs pull tasks of many items (every dim of every instance of a
//            batch) from a device counter, largest items first;
//   single - one item, task t = chunk t, one CTA per task (a per-dim refresh).
// The only waits are on the CTA's own MMA-completion mbarrier, each bounded: a wait
// that runs out sets TAPS_DEV_TIMEOUT, waits (bounded) once more for the MMAs issued,
// frees TMEM and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "taps_internal.cuh"

#define GT_THREADS 256
#define GT_MAXN 64     // modes and source terms of an item (each rounded up to 16)
#define GT_MAXOPS 4    // distinct operators of a dim
#define GT_SPIN (1u << 24)
#define GT_UNR 8       // loads in flight per thread

struct GtItem {
  const double* U;      // n x M, column-major (FP64 master)
  const double* band;   // [nops][n][2 hb + 1]
  const double* q;      // [Rf][n]
  double* gram;         // [nops][M][M]
  double* h;            // [Rf][M]
  double* partial;      // [ntasks][nops M M + Rf M] (items of several tasks)
  unsigned* ticket;     // one counter per item (items of several tasks)
  int n, M, hb, nops, Rf, ntasks;
};

struct GtTask {
  int item, c0, c1, slot;   // chunks [c0, c1) of the item; partial slot
};

// ---------------------------------------------------------------------------------
// PTX wrappers (tcgen05, mbarrier)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t gt_smem(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void gt_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gt_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ bool gt_mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = gt_smem(bar);
  for (uint32_t it = 0; it < GT_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// shared-memory matrix descriptor: start, leading / stride byte offsets, version 1, no swizzle
__device__ __forceinline__ uint64_t gt_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), A and B BF16
// (bits 7-9 and 10-12 = 1), both K-major, N >> 3 at bit 17, M = 128 (>> 4 at bit 24)
__device__ __forceinline__ uint32_t gt_idesc(int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}
__device__ __forceinline__ void gt_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void gt_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(gt_smem(bar))
               : "memory");
}
__device__ __forceinline__ void gt_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void gt_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 16 consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void gt_ld16(uint32_t taddr, float v[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// element offset of (row, k) in a K-major no-swizzle operand of `rows` rows: per K
// step of 16, row groups of 8 rows, two K cores of 8 elements (16 bytes) per group
__device__ __forceinline__ int gt_off(int rows, int row, int k) {
  return (k >> 4) * (rows * 16) + (row >> 3) * 128 + ((k >> 3) & 1) * 64 + (row & 7) * 8 + (k & 7);
}
// the operand as the contraction sees it: FP64 -> FP32 -> bfloat16 (round to nearest)
__device__ __forceinline__ __nv_bfloat16 gt_bf(double x) { return __float2bfloat16_rn((float)x); }

struct GtLayout {   // shared-memory carve-up of one launch (element offsets, bf16 / float)
  int N, NH, nops, rows;
};

// One task: chunks [c0, c1) of item `it` accumulated into TMEM at `tmem`.  Returns false
// after a timeout (the status word is set).
//
// Operand build of a chunk, division-free: warp w loads the factor rows of modes
// w, w + 8, ... (lane = row, coalesced along the column; 4 modes per pass), every
// thread loads its share
// of the chunk's band rows (one contiguous run per operator) and source rows, all loads
// of a thread issued before any is converted; the banded product is formed by thread
// (operator, row, slice of modes) with the row's band entries in registers.
#define GT_RPL(ROWS) (((ROWS) + 2 * (2 * TAPS_MAX_S + 1) + 31) / 32)   // factor rows per lane
template <int ROWS>
__device__ bool gt_task(const GtItem& it, int c0, int c1, const GtLayout& L, unsigned char* sm, uint32_t tmem,
                        uint64_t* mma_bar, uint32_t& phase, int* status) {
  constexpr int RPL = GT_RPL(ROWS);
  const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5, lane = tid & 31;
  const int M = it.M, n = it.n, hb = it.hb, nb = 2 * hb + 1, nops = it.nops, Rf = it.Rf;
  const int N = (M + 15) & ~15, NH = (Rf + 15) & ~15;
  const int RW = ROWS + 2 * hb;
  // carve-up: A [128 x ROWS], B [2 nops][N x ROWS], Bq [NH x ROWS] (bf16); Us, Bd (float)
  __nv_bfloat16* A = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* B = A + 128 * ROWS;
  __nv_bfloat16* Bq = B + 2 * L.nops * L.N * ROWS;
  float* Us = reinterpret_cast<float*>(Bq + L.NH * ROWS);
  float* Bd = Us + (ROWS + 2 * TAPS_MAX_S * 2 + 2) * (L.N + 1);
  const int ld = M + 1;
  const int nQ = NH * ROWS;               // source entries (padded terms)
  // mode slices of the banded product: thread (operator, row, slice)
  const int pairs = nops * ROWS;
  const int slices = pairs >= nt ? 1 : nt / pairs;
  const int per = (M + slices - 1) / slices;
  for (int c = c0; c < c1; ++c) {
    const int r0 = c * ROWS;
    const int rows_left = n - r0;          // rows of the chunk inside the dim
    // ---- loads: factor rows (8 modes per pass), band runs, source rows
    for (int m0 = warp; m0 < M; m0 += 8 * 4) {
      double v[4][RPL];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int m = m0 + 8 * a;
#pragma unroll
        for (int b = 0; b < RPL; ++b) {
          const int j = lane + 32 * b;
          const int g = r0 - hb + j;
          v[a][b] = (m < M && j < RW && g >= 0 && g < n) ? __ldg(it.U + (size_t)m * n + g) : 0.0;
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        const int m = m0 + 8 * a;
        if (m >= M) continue;
#pragma unroll
        for (int b = 0; b < RPL; ++b) {
          const int j = lane + 32 * b;
          if (j >= RW) continue;
          const __nv_bfloat16 x = gt_bf(v[a][b]);
          Us[j * ld + m] = __bfloat162float(x);
          const int i = j - hb;
          if (i >= 0 && i < ROWS) A[gt_off(128, m, i)] = x;
        }
      }
    }
    {
      // band rows: one contiguous run of ROWS * nb entries per operator (the chunk's
      // rows inside the dim loaded, the rest zero); source rows: NH x ROWS
      constexpr int BPT = (ROWS * (2 * (2 * TAPS_MAX_S + 1) + 1) + GT_THREADS - 1) / GT_THREADS;
      const int run = ROWS * nb, runv = min(rows_left, ROWS) * nb;
      for (int o = 0; o < nops; ++o) {
        const double* src = it.band + ((size_t)o * n + r0) * nb;
        double v[BPT];
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
          const int e = tid + u * GT_THREADS;
          v[u] = e < runv ? __ldg(src + e) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < BPT; ++u) {
          const int e = tid + u * GT_THREADS;
          if (e < run) Bd[o * run + e] = __bfloat162float(gt_bf(v[u]));
        }
      }
      constexpr int QPT = 4;
      for (int f0 = tid; f0 < nQ; f0 += GT_THREADS * QPT) {
        double v[QPT];
#pragma unroll
        for (int u = 0; u < QPT; ++u) {
          const int f = f0 + u * GT_THREADS;
          const int r = f / ROWS, i = f % ROWS;
          v[u] = (f < nQ && r < Rf && i < rows_left) ? __ldg(it.q + (size_t)r * n + r0 + i) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < QPT; ++u) {
          const int f = f0 + u * GT_THREADS;
          if (f < nQ) Bq[gt_off(NH, f / ROWS, f % ROWS)] = gt_bf(v[u]);
        }
      }
    }
    __syncthreads();
    // ---- Y_o = Op_o U for the chunk's rows (FP32), split into two bfloat16 parts
    for (int t = tid; t < pairs * slices; t += nt) {
      const int i = t % ROWS, rest = t / ROWS;
      const int o = rest % nops, sl = rest / nops;
      float br[2 * (2 * TAPS_MAX_S + 1) + 1];
      const float* brow = Bd + (o * ROWS + i) * nb;
#pragma unroll
      for (int k = 0; k < 2 * (2 * TAPS_MAX_S + 1) + 1; ++k) br[k] = k < nb ? brow[k] : 0.f;
      const int n0 = sl * per, n1 = min(N, n0 + per + (sl == slices - 1 ? N : 0));
      __nv_bfloat16* bh = B + (2 * o) * N * ROWS;
      __nv_bfloat16* bl = B + (2 * o + 1) * N * ROWS;
      for (int nn = n0; nn < n1; ++nn) {
        float y = 0.f;
        if (nn < M) {
          const float* ucol = Us + i * ld + nn;
#pragma unroll
          for (int k = 0; k < 2 * (2 * TAPS_MAX_S + 1) + 1; ++k)
            if (k < nb) y = fmaf(br[k], ucol[k * ld], y);
        }
        const __nv_bfloat16 hi = __float2bfloat16_rn(y);
        const __nv_bfloat16 lo = __float2bfloat16_rn(y - __bfloat162float(hi));
        const int off = gt_off(N, nn, i);
        bh[off] = hi;
        bl[off] = lo;
      }
    }
    // the generic-proxy writes above become visible to the tensor cores' async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      gt_fence_after();
      const uint32_t sa = gt_smem(A), sb = gt_smem(B), sq = gt_smem(Bq);
      const uint32_t id_n = gt_idesc(N), id_h = gt_idesc(NH);
      for (int ks = 0; ks < ROWS / 16; ++ks) {
        const uint64_t a = gt_desc(sa + (uint32_t)ks * 128u * 32u, 128, 256);
        const uint32_t first = (c == c0 && ks == 0) ? 0u : 1u;
        for (int o = 0; o < nops; ++o) {
          const uint32_t d = tmem + (uint32_t)(o * N);
          const uint32_t bh = sb + (uint32_t)((2 * o) * N * ROWS * 2) + (uint32_t)ks * (uint32_t)N * 32u;
          const uint32_t bl = sb + (uint32_t)((2 * o + 1) * N * ROWS * 2) + (uint32_t)ks * (uint32_t)N * 32u;
          gt_mma(d, a, gt_desc(bl, 128, 256), id_n, first);
          gt_mma(d, a, gt_desc(bh, 128, 256), id_n, 1u);
        }
        gt_mma(tmem + (uint32_t)(nops * N), a, gt_desc(sq + (uint32_t)ks * (uint32_t)NH * 32u, 128, 256), id_h,
               first);
      }
      gt_commit(mma_bar);
    }
    // every thread waits for the MMAs before the next chunk overwrites the operands;
    // the CTA agrees on the outcome so that all threads leave together
    const bool ok = __syncthreads_and(gt_mbar_wait(mma_bar, phase) ? 1 : 0) != 0;
    if (!ok) {   // `phase` stays the one still awaited, for the caller's final wait
      if (tid == 0) taps_flag(status, TAPS_DEV_TIMEOUT);
      return false;
    }
    phase ^= 1u;
    gt_fence_after();
  }
  return true;
}

// Epilogue of a task: the accumulators of the item's regions to `out` (FP64,
// [nops][M][M] then [Rf][M]); warps 0-3 read TMEM lanes 32 w .. 32 w + 31 (mode m).
__device__ void gt_store(const GtItem& it, uint32_t tmem, double* gout, double* hout) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp >= 4) return;
  const int M = it.M, N = (M + 15) & ~15, NH = (it.Rf + 15) & ~15;
  const int m = 32 * warp + lane;
  const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
  float v[16];
  for (int o = 0; o < it.nops; ++o)
    for (int c = 0; c < N; c += 16) {
      gt_ld16(lane_base + (uint32_t)(o * N + c), v);
      if (m < M)
        for (int j = 0; j < 16; ++j)
          if (c + j < M) gout[((size_t)o * M + m) * M + c + j] = (double)v[j];
    }
  for (int c = 0; c < NH; c += 16) {
    gt_ld16(lane_base + (uint32_t)(it.nops * N + c), v);
    if (m < M)
      for (int j = 0; j < 16; ++j)
        if (c + j < it.Rf) hout[(size_t)(c + j) * M + m] = (double)v[j];
  }
}

template <int ROWS>
__global__ void __launch_bounds__(GT_THREADS) gram_tc_kernel(const GtItem* __restrict__ items,
                                                             const GtTask* __restrict__ tasks, int ntasks,
                                                             unsigned* __restrict__ counter, GtItem single,
                                                             GtLayout L, int ncols, int* status) {
  extern __shared__ __align__(1024) unsigned char gt_sm[];
  __shared__ __align__(8) uint64_t mma_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_task, s_last;
  const int tid = threadIdx.x, warp = tid >> 5;
  taps_pdl_wait();
  unsigned char* sm = gt_sm + ((1024u - (gt_smem(gt_sm) & 1023u)) & 1023u);
  if (tid == 0) {
    gt_mbar_init(&mma_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(gt_smem(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  gt_fence_before();
  __syncthreads();
  gt_fence_after();
  const uint32_t tmem = tmem_slot;
  uint32_t phase = 0;
  bool ok = true;
  const bool queue = single.ntasks == 0;
  for (int pass = 0; ok; ++pass) {
    // the next task: from the queue, or this CTA's one chunk of the single item
    GtTask tk;
    if (queue) {
      if (tid == 0) s_task = (int)atomicAdd(counter, 1u);
      __syncthreads();
      const int t = s_task;
      if (t >= ntasks) break;
      tk = tasks[t];
    } else {
      if (pass > 0 || (int)blockIdx.x >= single.ntasks) break;
      tk.item = 0;
      tk.c0 = blockIdx.x;
      tk.c1 = blockIdx.x + 1;
      tk.slot = blockIdx.x;
    }
    const GtItem it = queue ? items[tk.item] : single;
    ok = gt_task<ROWS>(it, tk.c0, tk.c1, L, sm, tmem, &mma_bar, phase, status);
    if (!ok) break;
    const size_t stride = (size_t)it.nops * it.M * it.M + (size_t)it.Rf * it.M;
    if (it.ntasks == 1) {
      gt_store(it, tmem, it.gram, it.h);
    } else {
      double* p = it.partial + (size_t)tk.slot * stride;
      gt_store(it, tmem, p, p + (size_t)it.nops * it.M * it.M);
    }
    gt_fence_before();
    __threadfence();
    __syncthreads();
    if (it.ntasks > 1) {
      // the last task of the item sums the partials in task order
      if (tid == 0) s_last = (atomicAdd(it.ticket, 1u) == (unsigned)it.ntasks - 1u) ? 1 : 0;
      __syncthreads();
      if (s_last) {
        __threadfence();
        for (size_t e = tid; e < stride; e += blockDim.x) {
          double s = 0.0;
          for (int t = 0; t < it.ntasks; ++t) s += __ldcg(it.partial + (size_t)t * stride + e);
          const size_t g = (size_t)it.nops * it.M * it.M;
          if (e < g) it.gram[e] = s;
          else it.h[e - g] = s;
        }
        if (tid == 0) *it.ticket = 0u;   // ready for the next launch
      }
    }
    __syncthreads();   // s_task / s_last and TMEM are reused by the next task
    gt_fence_after();
  }
  if (!ok) {   // MMAs may still be in flight: wait (bounded) before releasing TMEM
    gt_mbar_wait(&mma_bar, phase);
  }
  gt_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
static size_t gt_smem_bytes(const GtLayout& L) {
  const size_t bf = (size_t)(128 + 2 * L.nops * L.N + L.NH) * L.rows * 2;
  const size_t fl = (size_t)(L.rows + 2 * TAPS_MAX_S * 2 + 2) * (L.N + 1) + (size_t)L.nops * L.rows * (2 * (2 * TAPS_MAX_S + 1) + 1);
  return 1024 + bf + fl * 4;
}
static int gt_cols(const GtLayout& L) {
  const int need = L.nops * L.N + L.NH;
  int c = 32;
  while (c < need) c <<= 1;
  return c;
}

int taps_gram_tc_eligible(int M, int nops, int Rf, int hb) {
  return M >= 1 && M <= GT_MAXN && nops >= 1 && nops <= GT_MAXOPS && Rf >= 1 && Rf <= GT_MAXN && hb >= 0 &&
         hb <= 2 * TAPS_MAX_S + 1;
}

int taps_gram_tc_setup(int maxsm) {
  TAPS_CUDA(cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - 1024));
  TAPS_CUDA(cudaFuncSetAttribute(gram_tc_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, maxsm - 1024));
  return TAPS_OK;
}

// One item split into one task per chunk of `rows`, one CTA each (the per-dim refresh
// of a sweep): partials in `partial`, the item's ticket in `ticket` (zero on entry,
// left zero).
int taps_gram_tc_single(const double* U, const double* band, const double* q, double* gram, double* h, int n,
                        int M, int hb, int nops, int Rf, double* partial, unsigned* ticket, int rows,
                        cudaStream_t s, int* status) {
  if (!taps_gram_tc_eligible(M, nops, Rf, hb) || (rows != 64 && rows != 128)) return TAPS_ERR_INVALID_ARG;
  GtItem it;
  it.U = U;
  it.band = band;
  it.q = q;
  it.gram = gram;
  it.h = h;
  it.partial = partial;
  it.ticket = ticket;
  it.n = n;
  it.M = M;
  it.hb = hb;
  it.nops = nops;
  it.Rf = Rf;
  it.ntasks = (n + rows - 1) / rows;
  GtLayout L;
  L.N = (M + 15) & ~15;
  L.NH = (Rf + 15) & ~15;
  L.nops = nops;
  L.rows = rows;
  const size_t smem = gt_smem_bytes(L);
  const int ncols = gt_cols(L);
  if (rows == 64)
    TAPS_CUDA(taps_launch_pdl(gram_tc_kernel<64>, dim3(it.ntasks), dim3(GT_THREADS), smem, s,
                              (const GtItem*)nullptr, (const GtTask*)nullptr, 0, (unsigned*)nullptr, it, L, ncols,
                              status));
  else
    TAPS_CUDA(taps_launch_pdl(gram_tc_kernel<128>, dim3(it.ntasks), dim3(GT_THREADS), smem, s,
                              (const GtItem*)nullptr, (const GtTask*)nullptr, 0, (unsigned*)nullptr, it, L, ncols,
                              status));
  return TAPS_OK;
}

// Many items in one persistent launch (queue mode).  The host lists items (device
// pointers filled in), builds the tasks (`cpt` chunks each, items by decreasing
// size), copies both into `dev_buf` (at least taps_gram_tc_queue_bytes) and launches
// `ctas` CTAs.  Item partials go to `partial` (taps_gram_tc_partial_doubles), tickets
// to `tickets` (one per item, zero on entry, left zero).
size_t taps_gram_tc_queue_bytes(int nitems, int max_tasks) {
  return sizeof(GtItem) * (size_t)nitems + sizeof(GtTask) * (size_t)max_tasks + 64;
}

int taps_gram_tc_queue(const std::vector<GtHostItem>& hitems, int rows, int cpt, int ctas, void* dev_buf,
                       size_t dev_buf_bytes, double* partial, size_t partial_doubles, unsigned* tickets,
                       cudaStream_t s, int* status, double* flops_out, double* bytes_out, cudaEvent_t ev0,
                       cudaEvent_t ev1) {
  if (hitems.empty() || (rows != 64 && rows != 128) || cpt < 1 || ctas < 1) return TAPS_ERR_INVALID_ARG;
  std::vector<int> order(hitems.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
  auto cost = [&](int i) {
    const GtHostItem& h = hitems[i];
    return (double)h.n * ((double)h.M * (8 + 8 * (2 * h.hb + 1) * h.nops) + 8.0 * h.Rf);
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  std::vector<GtItem> items(hitems.size());
  std::vector<GtTask> tasks;
  GtLayout L;
  L.N = 16;
  L.NH = 16;
  L.nops = 1;
  L.rows = rows;
  size_t poff = 0;
  double fl = 0.0, by = 0.0;
  for (size_t k = 0; k < order.size(); ++k) {
    const int i = order[k];
    const GtHostItem& h = hitems[i];
    if (!taps_gram_tc_eligible(h.M, h.nops, h.Rf, h.hb)) return TAPS_ERR_INVALID_ARG;
    GtItem& it = items[k];
    it.U = h.U;
    it.band = h.band;
    it.q = h.q;
    it.gram = h.gram;
    it.h = h.h;
    it.n = h.n;
    it.M = h.M;
    it.hb = h.hb;
    it.nops = h.nops;
    it.Rf = h.Rf;
    const int nch = (h.n + rows - 1) / rows;
    it.ntasks = (nch + cpt - 1) / cpt;
    it.ticket = tickets + k;
    const size_t stride = (size_t)h.nops * h.M * h.M + (size_t)h.Rf * h.M;
    it.partial = partial + poff;
    if (it.ntasks > 1) poff += stride * it.ntasks;
    for (int t = 0; t < it.ntasks; ++t) {
      GtTask tk;
      tk.item = (int)k;
      tk.c0 = t * cpt;
      tk.c1 = std::min(nch, (t + 1) * cpt);
      tk.slot = t;
      tasks.push_back(tk);
    }
    L.N = std::max(L.N, (h.M + 15) & ~15);
    L.NH = std::max(L.NH, (h.Rf + 15) & ~15);
    L.nops = std::max(L.nops, h.nops);
    const int nb = 2 * h.hb + 1;
    fl += h.nops * (2.0 * nb * h.n * h.M + 2.0 * h.n * (double)h.M * h.M) + 2.0 * h.Rf * h.n * h.M;
    by += 8.0 * ((double)h.n * h.M + (double)h.nops * h.n * nb + (double)h.Rf * h.n + (double)h.nops * h.M * h.M +
                 (double)h.Rf * h.M);
  }
  if (poff > partial_doubles) return TAPS_ERR_INVALID_ARG;
  const size_t need = taps_gram_tc_queue_bytes((int)items.size(), (int)tasks.size());
  if (need > dev_buf_bytes) return TAPS_ERR_INVALID_ARG;
  unsigned char* base = (unsigned char*)dev_buf;
  unsigned* counter = (unsigned*)base;
  GtItem* ditems = (GtItem*)(base + 64);
  GtTask* dtasks = (GtTask*)(base + 64 + sizeof(GtItem) * items.size());
  TAPS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
  TAPS_CUDA(cudaMemcpyAsync(ditems, items.data(), sizeof(GtItem) * items.size(), cudaMemcpyHostToDevice, s));
  TAPS_CUDA(cudaMemcpyAsync(dtasks, tasks.data(), sizeof(GtTask) * tasks.size(), cudaMemcpyHostToDevice, s));
  GtItem none;
  memset(&none, 0, sizeof(none));
  const size_t smem = gt_smem_bytes(L);
  const int ncols = gt_cols(L);
  if (ev0) TAPS_CUDA(cudaEventRecord(ev0, s));
  if (rows == 64)
    gram_tc_kernel<64><<<ctas, GT_THREADS, smem, s>>>(ditems, dtasks, (int)tasks.size(), counter, none, L, ncols,
                                                      status);
  else
    gram_tc_kernel<128><<<ctas, GT_THREADS, smem, s>>>(ditems, dtasks, (int)tasks.size(), counter, none, L, ncols,
                                                       status);
  TAPS_CUDA(cudaGetLastError());
  if (ev1) TAPS_CUDA(cudaEventRecord(ev1, s));
  // the host arrays are copied from pageable memory: wait for the copies before they go
  TAPS_CUDA(cudaStreamSynchronize(s));
  if (flops_out) *flops_out = fl;
  if (bytes_out) *bytes_out = by;
  return TAPS_OK;
}

// Dynamic shared memory and TMEM columns of a queue launch (for the tuner's
// occupancy choice).
int taps_gram_tc_footprint(int rows, int maxN, int maxNH, int maxops, size_t* smem, int* ncols) {
  GtLayout L;
  L.N = maxN;
  L.NH = maxNH;
  L.nops = maxops;
  L.rows = rows;
  *smem = gt_smem_bytes(L);
  *ncols = gt_cols(L);
  return TAPS_OK;
}
