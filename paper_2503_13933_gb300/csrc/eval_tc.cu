// Full-grid reconstruction on the 5th-generation tensor cores (Eq. 13 at nodes).
//
// The reconstruction is the rank-M product out[r][c] = sum_m A[r][m] B[c][m] (A: the
// row-wise products of the leading dims' factor rows, B: those of the trailing dims),
// a GEMM with a short contraction (K = M) and a large FP32 output.  With K ~ 30 the
// output stream costs ~0.3 ms per 2 GB on HBM3e while the FP32 FMAs on the CUDA cores
// cost ~0.45 ms, so the product goes to tcgen05: per 128 x 256 output tile the
// accumulator lives in tensor memory (TMEM), the operands are staged in shared memory
// by bulk copies and the four epilogue warps stream the tile out.
//
// Precision: kind::tf32 keeps 10 mantissa bits of each operand.  Every FP32 operand
// x is split as x = hi + lo with hi = x with its 13 low mantissa bits cleared (exact
// in TF32) and lo = x - hi (exact in FP32), and the product is accumulated in FP32
// as hi*hi + hi*lo + lo*hi (the lo*lo term is below 2^-22 relative).  This keeps the
// FP32 reconstruction within a few 1e-7 of the FP32-operand product.
//
// Roles in one persistent CTA per SM (320 threads):
//   warp 0       : bulk-copy producer (one elected lane) and TMEM allocation
//   warp 1       : MMA issuer (one elected lane)
//   warps 2 - 9  : epilogue; warp w reads TMEM lanes 32 (w % 4) .. 32 (w % 4) + 31 and
//                  the column half (w - 2) / 4 of the tile
// Two TMEM accumulators (256 columns each, 512 in all) let the operand copy and the
// MMAs of the next tile run while the previous tile streams out.  Up to K = 32 the copy
// and the MMAs are short next to a tile's 128 KB output, so a tile's operands travel in
// one stage and the rest of the shared memory goes to the epilogue's staging blocks;
// beyond (up to K = 128) the operands of a tile travel in chunks of 16 K through three
// stages, the accumulator collecting the chunks' MMAs.  Every wait on an mbarrier is bounded;
// a wait that runs out sets TAPS_DEV_TIMEOUT, the other roles see the abort flag, the
// MMA issuer waits (bounded) for its outstanding MMAs, and TMEM is freed on exit.
#include <stdint.h>

#include <algorithm>

#include "taps_internal.cuh"

#define TC_BM 128                    // output rows per tile (TMEM lanes)
#define TC_BN 256                    // output columns per tile (TMEM columns)
#define TC_KSTEP 8                   // K of one kind::tf32 MMA
#define TC_MAXK 128                  // largest padded K handled here (M <= 128)
#define TC_A_KBLK (TC_BM * TC_KSTEP) // floats of one A K-step block (4 KB)
#define TC_B_KBLK (TC_BN * TC_KSTEP) // floats of one B K-step block (8 KB)
#define TC_MAXSTAGES 3               // operand stages: 1 for K <= 32 (a tile's operands in one
                                     // stage), 3 stages of 16 K each beyond
#define TC_ACC 2                     // TMEM accumulators
#define TC_EPI_WARPS 8               // two per TMEM lane quarter, one per column half
#define TC_THREADS (64 + 32 * TC_EPI_WARPS)
#define TC_SPIN (1u << 24)

// ---------------------------------------------------------------------------------
// Operand images.  An operand block of `rows` rows (128 for A, 256 for B) is stored
// as [hi | lo][K-step][row group of 8][K core of 4 floats][row in group][4 floats]:
// the no-swizzle K-major layout of the MMA, with core matrices of 8 rows x 16 bytes,
// 128 bytes between the two K cores of a row group (leading byte offset) and 256
// bytes between row groups (stride byte offset).  One block is one contiguous run of
// 2 * ksteps * rows * 8 floats, so a tile's operands arrive by plain bulk copies.
// ---------------------------------------------------------------------------------
__device__ __forceinline__ size_t tc_img_offset(int rows, int ksteps, int row, int k, int part) {
  const int ks = k >> 3, kk = k & 7;
  return ((size_t)part * ksteps + ks) * ((size_t)rows * TC_KSTEP) + (size_t)(row >> 3) * 64 +
         (kk >> 2) * 32 + (row & 7) * 4 + (kk & 3);
}

// Image of X[x][m] = prod_{d in [d0, d1)} G_d[i_d(x)][m] (x in C order over d0..d1-1),
// rows padded to a multiple of `rows`, m padded with zeros to 8 * ksteps.  One thread
// per (row, 4 consecutive m): the row's indices are decomposed once (32-bit when the
// row count allows) and the 4 hi and 4 lo values go out as two 16-byte stores, which
// for 8 consecutive rows fill one 128-byte core-matrix row group.
__global__ void tc_image_kernel(const float* __restrict__ G, GridSpec gs, int d0, int d1, int M, int ksteps,
                                long long nx, int rows, float* __restrict__ img) {
  const int kq = ksteps * TC_KSTEP / 4;
  const long long nblk = (nx + rows - 1) / rows;
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nblk * rows * kq) return;
  // consecutive threads take consecutive rows (coalesced 16-byte stores)
  const long long padded = nblk * rows;
  const int q = (int)(idx / padded);
  const long long x = idx - (long long)q * padded;
  long long off[TAPS_MAX_DIMS];
  bool in = x < nx;
  if (in) {
    if (nx < (1ll << 31)) {
      unsigned y = (unsigned)x;
#pragma unroll
      for (int d = TAPS_MAX_DIMS - 1; d >= 0; --d) {
        off[d] = 0;
        if (d >= d0 && d < d1) {
          const unsigned c = (unsigned)gs.count[d], qq = y / c;
          off[d] = gs.goff[d] + (long long)(y - qq * c) * M;
          y = qq;
        }
      }
    } else {
      long long y = x;
#pragma unroll
      for (int d = TAPS_MAX_DIMS - 1; d >= 0; --d) {
        off[d] = 0;
        if (d >= d0 && d < d1) {
          const long long qq = y / gs.count[d];
          off[d] = gs.goff[d] + (y - qq * gs.count[d]) * M;
          y = qq;
        }
      }
    }
  }
  float hi[4], lo[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = 4 * q + j;
    float v = 0.f;
    if (in && m < M) {
      v = 1.f;
#pragma unroll
      for (int d = 0; d < TAPS_MAX_DIMS; ++d)
        if (d >= d0 && d < d1) v *= G[off[d] + m];
    }
    hi[j] = __uint_as_float(__float_as_uint(v) & 0xFFFFE000u);
    lo[j] = v - hi[j];
  }
  const long long blk = x / rows;
  const int row = (int)(x - blk * rows);
  float* base = img + (size_t)blk * 2 * ksteps * rows * TC_KSTEP;
  *reinterpret_cast<float4*>(base + tc_img_offset(rows, ksteps, row, 4 * q, 0)) =
      make_float4(hi[0], hi[1], hi[2], hi[3]);
  *reinterpret_cast<float4*>(base + tc_img_offset(rows, ksteps, row, 4 * q, 1)) =
      make_float4(lo[0], lo[1], lo[2], lo[3]);
}

// ---------------------------------------------------------------------------------
// PTX wrappers
// ---------------------------------------------------------------------------------
__device__ __forceinline__ uint32_t tc_smem(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void tc_mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tc_smem(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void tc_mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(tc_smem(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tc_mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(tc_smem(bar)) : "memory");
}
// Waits for the completion of the phase with parity `parity`; false on timeout or
// when another role has aborted.
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  const uint32_t a = tc_smem(bar);
  for (uint32_t it = 0; it < TC_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (*abort_flag) return false;
  }
  return false;
}
__device__ __forceinline__ void tc_bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          tc_smem(dst)),
      "l"(src), "r"(bytes), "r"(tc_smem(bar))
      : "memory");
}
// Shared-memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::tf32: FP32 accumulator (bits 4-5 = 1), A and B
// TF32 (bits 7-9 and 10-12 = 2), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(TC_BN >> 3) << 17) |
                              ((uint32_t)(TC_BM >> 4) << 24);

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(TC_IDESC), "r"(accumulate));
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   tc_smem(bar))
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// 32 consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float v[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// ---------------------------------------------------------------------------------
// The persistent kernel.  Tile t covers rows 128 (t % nrb) .. and columns 256 (t / nrb)
// .. (column-block-major, so that consecutive tiles share the B block in L2), or, with
// rowmajor (an A image too large for L2), rows 128 (t / ncb) .. and columns
// 256 (t % ncb) .., so that the column blocks of one row block run together.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(TC_THREADS, 1) eval_tc_kernel(const float* __restrict__ Aimg,
                                                                 const float* __restrict__ Bimg,
                                                                 long long R, int C, int ksteps, int kc, int nst,
                                                                 float* __restrict__ out, int vec_ok,
                                                                 int rowmajor, int* status) {
  extern __shared__ __align__(1024) unsigned char tc_sm[];
  __shared__ __align__(8) uint64_t full_bar[TC_MAXSTAGES], empty_bar[TC_MAXSTAGES];
  __shared__ __align__(8) uint64_t acc_full[TC_ACC], acc_empty[TC_ACC], drain_bar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long nrb = (R + TC_BM - 1) / TC_BM;
  const long long ncb = (C + TC_BN - 1) / TC_BN;
  const long long ntiles = nrb * ncb;
  // an operand block in global memory: [hi | lo][ksteps][rows x 8 floats]; a stage
  // holds one K chunk of kc steps of both operands: [A hi][A lo][B hi][B lo], each part
  // kc steps long (with kc = ksteps, one chunk: a tile's whole operands)
  const uint32_t a_bytes = 2u * ksteps * TC_A_KBLK * 4u;
  const uint32_t b_bytes = 2u * ksteps * TC_B_KBLK * 4u;
  const uint32_t stage_bytes = 2u * kc * (TC_A_KBLK + TC_B_KBLK) * 4u;
  const int nchunks = (ksteps + kc - 1) / kc;
  // 1024-byte aligned stages
  unsigned char* base = tc_sm + ((1024u - (tc_smem(tc_sm) & 1023u)) & 1023u);

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < nst; ++s) {
      tc_mbar_init(&full_bar[s], 1);
      tc_mbar_init(&empty_bar[s], 1);
    }
    for (int b = 0; b < TC_ACC; ++b) {
      tc_mbar_init(&acc_full[b], 1);
      tc_mbar_init(&acc_empty[b], TC_EPI_WARPS);
    }
    tc_mbar_init(&drain_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc_smem(&tmem_slot)),
                 "r"(TC_ACC * TC_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0) {
    if (lane == 0) {   // ---- producer: one stage per K chunk of a tile
      long long i = 0;   // chunks issued
      bool stop = false;
      for (long long t = blockIdx.x; t < ntiles && !stop; t += gridDim.x) {
        const long long rb = rowmajor ? t / ncb : t % nrb, cb = rowmajor ? t % ncb : t / nrb;
        const unsigned char* asrc = (const unsigned char*)Aimg + (size_t)rb * a_bytes;
        const unsigned char* bsrc = (const unsigned char*)Bimg + (size_t)cb * b_bytes;
        for (int c = 0; c < nchunks; ++c, ++i) {
          const int s = (int)(i % nst);
          const uint32_t ph = (uint32_t)((i / nst) & 1);
          if (!tc_mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag)) {
            abort_flag = 1;
            taps_flag(status, TAPS_DEV_TIMEOUT);
            stop = true;
            break;
          }
          const int k0 = c * kc, kcc = min(kc, ksteps - k0);
          unsigned char* st = base + (size_t)s * stage_bytes;
          tc_mbar_expect_tx(&full_bar[s], 2u * kcc * (TC_A_KBLK + TC_B_KBLK) * 4u);
          // (part, source offset, stage offset, bytes) of the chunk's four parts
          const uint32_t abk = TC_A_KBLK * 4u, bbk = TC_B_KBLK * 4u;
          const unsigned char* src[4] = {asrc + (size_t)k0 * abk, asrc + (size_t)(ksteps + k0) * abk,
                                         bsrc + (size_t)k0 * bbk, bsrc + (size_t)(ksteps + k0) * bbk};
          const uint32_t dst[4] = {0u, (uint32_t)kc * abk, 2u * kc * abk, 2u * kc * abk + (uint32_t)kc * bbk};
          const uint32_t len[4] = {(uint32_t)kcc * abk, (uint32_t)kcc * abk, (uint32_t)kcc * bbk,
                                   (uint32_t)kcc * bbk};
          for (int part = 0; part < 4; ++part)
            for (uint32_t o = 0; o < len[part]; o += 8192u)
              tc_bulk_g2s(st + dst[part] + o, src[part] + o, min(8192u, len[part] - o), &full_bar[s]);
        }
      }
      // copies still in flight land before the CTA leaves: wait for the stages issued
      // but not consumed (bounded)
      if (abort_flag) {
        const long long issued = i;
        for (long long j = (issued > nst ? issued - nst : 0); j < issued; ++j) {
          volatile int never = 0;
          tc_mbar_wait(&full_bar[j % nst], (uint32_t)((j / nst) & 1), (volatile int*)&never);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // ---- MMA issuer
      long long i = 0, tile = 0;   // chunks consumed, tiles started
      bool stop = false;
      for (long long t = blockIdx.x; t < ntiles && !stop; t += gridDim.x, ++tile) {
        const int b = (int)(tile % TC_ACC);
        const uint32_t pb = (uint32_t)((tile / TC_ACC) & 1);
        if (!tc_mbar_wait(&acc_empty[b], pb ^ 1u, &abort_flag)) {
          abort_flag = 1;
          taps_flag(status, TAPS_DEV_TIMEOUT);
          break;
        }
        const uint32_t d = tmem + (uint32_t)(b * TC_BN);
        uint32_t acc = 0;
        for (int c = 0; c < nchunks; ++c, ++i) {
          const int s = (int)(i % nst);
          const uint32_t ph = (uint32_t)((i / nst) & 1);
          if (!tc_mbar_wait(&full_bar[s], ph, &abort_flag)) {
            abort_flag = 1;
            taps_flag(status, TAPS_DEV_TIMEOUT);
            stop = true;
            break;
          }
          tc_fence_after();
          const int kcc = min(kc, ksteps - c * kc);
          const uint32_t sa = tc_smem(base + (size_t)s * stage_bytes);
          const uint32_t sb = sa + 2u * kc * TC_A_KBLK * 4u;
          // lo * hi, hi * lo, then hi * hi: the small terms first (within the chunk)
          for (int k = 0; k < kcc; ++k) {
            const uint32_t a_hi = sa + (uint32_t)k * TC_A_KBLK * 4u;
            const uint32_t a_lo = a_hi + (uint32_t)kc * TC_A_KBLK * 4u;
            const uint32_t b_hi = sb + (uint32_t)k * TC_B_KBLK * 4u;
            const uint32_t b_lo = b_hi + (uint32_t)kc * TC_B_KBLK * 4u;
            tc_mma(d, tc_desc(a_lo, 128, 256), tc_desc(b_hi, 128, 256), acc);
            acc = 1;
            tc_mma(d, tc_desc(a_hi, 128, 256), tc_desc(b_lo, 128, 256), acc);
          }
          for (int k = 0; k < kcc; ++k) {
            const uint32_t a_hi = sa + (uint32_t)k * TC_A_KBLK * 4u;
            const uint32_t b_hi = sb + (uint32_t)k * TC_B_KBLK * 4u;
            tc_mma(d, tc_desc(a_hi, 128, 256), tc_desc(b_hi, 128, 256), 1u);
          }
          tc_commit(&empty_bar[s]);   // operands free once these MMAs have read them
        }
        if (stop) break;
        tc_commit(&acc_full[b]);    // accumulator ready for the epilogue
      }
      // every MMA issued by this thread has completed before TMEM is released
      tc_commit(&drain_bar);
      volatile int never = 0;
      if (!tc_mbar_wait(&drain_bar, 0u, (volatile int*)&never)) taps_flag(status, TAPS_DEV_TIMEOUT);
    }
  } else {   // ---- epilogue: warps 2..9
    const int q = warp & 3;             // TMEM lane quarter of this warp
    const int half = (warp - 2) >> 2;   // column half of the tile
    // 32 x 32 block of this warp, row stride 36 floats: the row-wise float4 writes and
    // the column-wise float4 reads of 8 lanes at a time fall in distinct banks
    float* tb = reinterpret_cast<float*>(base + (size_t)nst * stage_bytes) + (warp - 2) * (32 * 36);
    const int rr = lane >> 3, c4 = (lane & 7) * 4;   // store pattern: 4 rows x 8 float4
    long long i = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int b = (int)(i % TC_ACC);
      const uint32_t pb = (uint32_t)((i / TC_ACC) & 1);
      if (!tc_mbar_wait(&acc_full[b], pb, &abort_flag)) {
        abort_flag = 1;
        taps_flag(status, TAPS_DEV_TIMEOUT);
        break;
      }
      tc_fence_after();
      const long long rb = rowmajor ? t / ncb : t % nrb, cb = rowmajor ? t % ncb : t / nrb;
      const long long row0 = rb * TC_BM + 32 * q;
      const int c0 = (int)(cb * TC_BN) + half * (TC_BN / 2);
      const uint32_t tbase = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * TC_BN + half * (TC_BN / 2));
#pragma unroll 1
      for (int ch = 0; ch < TC_BN / 64; ++ch) {
        float v[32];
        tc_ld32(tbase + (uint32_t)(32 * ch), v);   // lane = row, 32 consecutive columns
#pragma unroll
        for (int j = 0; j < 32; j += 4)
          *reinterpret_cast<float4*>(tb + lane * 36 + j) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
        __syncwarp();
        const int cc = c0 + 32 * ch + c4;
#pragma unroll
        for (int k = 0; k < 8; ++k) {   // rows rr, rr + 4, ..., each by 8 lanes x 16 bytes
          const int r = rr + 4 * k;
          const long long row = row0 + r;
          const float4 w = *reinterpret_cast<const float4*>(tb + r * 36 + c4);
          if (row < R) {
            float* o = out + row * (long long)C + cc;
            if (vec_ok && cc + 4 <= C) {
              __stcs(reinterpret_cast<float4*>(o), w);
            } else {
              if (cc < C) __stcs(o, w.x);
              if (cc + 1 < C) __stcs(o + 1, w.y);
              if (cc + 2 < C) __stcs(o + 2, w.z);
              if (cc + 3 < C) __stcs(o + 3, w.w);
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) tc_mbar_arrive(&acc_empty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_ACC * TC_BN)
                 : "memory");
}

// ---------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------
size_t taps_eval_tc_scratch(long long rows, long long cols, int M) {
  const int ksteps = (M + TC_KSTEP - 1) / TC_KSTEP;
  const long long nrb = (rows + TC_BM - 1) / TC_BM, ncb = (cols + TC_BN - 1) / TC_BN;
  return sizeof(float) * 2 * (size_t)ksteps * TC_KSTEP * ((size_t)nrb * TC_BM + (size_t)ncb * TC_BN);
}

int taps_eval_tc_usable(long long rows, long long cols, int M) {
  return M >= 1 && M <= TC_MAXK && rows >= TC_BM && cols >= 128 && cols <= (1ll << 30);
}

int taps_eval_tc_setup(int maxsm) { return taps_allow_dyn_smem((const void*)eval_tc_kernel, maxsm); }

int taps_eval_tc(taps_problem* P, const float* G, const GridSpec& gs, int split, int M, long long rows,
                 long long cols, void* scratch, float* out) {
  const int ksteps = (M + TC_KSTEP - 1) / TC_KSTEP;
  const long long nrb = (rows + TC_BM - 1) / TC_BM, ncb = (cols + TC_BN - 1) / TC_BN;
  float* Aimg = (float*)scratch;
  float* Bimg = Aimg + 2 * (size_t)ksteps * TC_KSTEP * nrb * TC_BM;
  cudaStream_t s = P->stream;
  const long long na = nrb * TC_BM * ksteps * TC_KSTEP / 4, nb = ncb * TC_BN * ksteps * TC_KSTEP / 4;
  tc_image_kernel<<<(unsigned)((na + 255) / 256), 256, 0, s>>>(G, gs, 0, split, M, ksteps, rows, TC_BM, Aimg);
  tc_image_kernel<<<(unsigned)((nb + 255) / 256), 256, 0, s>>>(G, gs, split, gs.D, M, ksteps, cols, TC_BN,
                                                              Bimg);
  // K <= 32: a tile's operands in one stage; beyond, three stages of 2 K steps (16 K)
  const int kc = ksteps <= 4 ? ksteps : 2, nst = ksteps <= 4 ? 1 : TC_MAXSTAGES;
  const size_t stage = (size_t)2 * kc * (TC_A_KBLK + TC_B_KBLK) * sizeof(float);
  const size_t smem = nst * stage + TC_EPI_WARPS * 32 * 36 * sizeof(float) + 1024;
  const long long ntiles = nrb * ncb;
  const int grid = (int)std::min<long long>(ntiles, P->num_sms);
  const int vec_ok = ((cols & 3) == 0 && (((uintptr_t)out) & 15) == 0) ? 1 : 0;
  // the larger operand image is walked in the outer order, so that each of its blocks
  // is read from HBM once and its neighbours' tiles find it in L2
  const int rowmajor = (nrb * TC_BM > ncb * TC_BN) && nrb * TC_BM * 2ll * ksteps * TC_KSTEP * 4 > (32ll << 20);
  eval_tc_kernel<<<grid, TC_THREADS, smem, s>>>(Aimg, Bimg, rows, (int)cols, ksteps, kc, nst, out, vec_ok,
                                                 rowmajor, P->d_status);
  TAPS_CUDA(cudaGetLastError());
  return TAPS_OK;
}
