// Complex64 block products with 9 to 32 right-hand sides on the tcgen05 tensor
// cores (the multi-RHS matrix-vector products of GMRES on Eq. finalsystem, one
// pass over the stored blocks per step).
//
// Complex product as one real GEMM.  A complex64 row-major block A (m x n) is,
// byte for byte, a row-major FP32 matrix A' of m rows and 2n columns (re, im
// interleaved).  With B' (2n x 64) holding, for right-hand side r, the columns
//     B'[2c, 2r] = Re x_r[c],  B'[2c+1, 2r] = -Im x_r[c]
//     B'[2c, 2r+1] = Im x_r[c], B'[2c+1, 2r+1] = Re x_r[c],
// D = A' B' holds Re y_r in column 2r and Im y_r in column 2r+1.  A' is the
// stored block itself (the MMA's K-major A operand, streamed by TMA); B' (hi and
// lo, below) is built for every K chunk of every job once per pass by
// tc_bprime_kernel into global memory and streamed by TMA as well (it is the same
// for all row tiles of a job, so building it in each tile would repeat the work).
//
// Near-FP32 accuracy from TF32 operands (three products): with hi(v) = v rounded
// to TF32 (10 stored mantissa bits: |v - hi| <= 2^-11 |v|) and lo(v) = v - hi
// rounded to TF32 (error <= 2^-11 |v - hi| <= 2^-22 |v|),
//     D = hi(A) hi(B) + lo(A) hi(B) + hi(A) lo(B)        (FP32 accumulation),
// the dropped lo(A) lo(B) (<= 2^-22 |A||B|) and the two roundings of lo leave
// each product term within 3 x 2^-22 of |A||B| (about 2^-22 for typical data),
// against 2^-24 for an FP32 product; the sums are compensated (below).
//
// Per CTA (one per SM, persistent over its tiles, longest first), 128-row
// tiles streamed in stages of 4 TMA boxes (128 rows x 4 x 128 B, 128-byte
// swizzled): 512 contiguous bytes of every row per stage, which DRAM serves at
// ~0.98 of the copy rate, against ~0.65 for 128-byte runs.  Each stage is
// split into four K sub-chunks of 32 FP32 columns.  Warp-specialised,
// synchronised by mbarriers only:
//   warp 0   TMA: a ring of 2 stages (128 KB in flight per SM);
//   warp 18  TMA: B' hi/lo of each sub-chunk (one 128-row x 128 B box) into the
//            operand buffer of that sub-chunk once the MMAs that read it before
//            have completed;
//   warps 2-9 split (two per TMEM lane quarter, half the K columns each):
//            thread = row; for each sub-chunk reads its row, splits it
//            into hi and lo and stores both into a TMEM operand buffer (A of
//            the MMA in tensor memory: lane = row, column = K); the ring stage is
//            freed after its fourth sub-chunk;
//   warp 1   MMA: one thread issues 8 MMAs per sub-chunk, per K step of 8:
//            hi(A) x [hi(B') | lo(B')] (M 128, N 128: B' hi and lo are the two
//            halves of one 128-row operand) and lo(A) x hi(B') (N 64) into the
//            first half, into one of two 128-column TMEM accumulators, a fresh
//            one for every stage (a segment of 128 K columns), and commits them
//            to the operand buffer's barrier.  Two products per K step instead
//            of three N = 64 ones: the tensor pipe spends ~70 cycles on an
//            M 128 N 64 K 8 TF32 product, so three of them per K step took more
//            of its time than the stage's HBM transfer leaves;
//   warps 10-17 epilogue: fold each segment's accumulator (the sum of its two
//            halves) into compensated FP32 sums in registers (warp w: TMEM
//            lanes 32 (w % 4) .., 32 of the 64 output columns), and at the end
//            of a tile write Y.
// The tensor core rounds its FP32 accumulator at every MMA: a tile's ~10^4
// MMAs into one accumulator would lose ~2^-17 of the result; segments of 32
// MMAs and compensated sums across them keep the product as accurate as an
// FP32 CUDA-core product.
// Operand buffers: 4 for A (TMEM, the most that fits beside the two 128-column
// accumulators), 6 for B' (shared memory), so that the B' loads, whose latency
// from L2 under the streaming load is ~10^3 cycles, are issued well ahead.
// Tiles are padded to whole stages (zero columns from TMA and zero B').
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <queue>

#include "gemm_tc.h"

namespace sldm {

namespace {

constexpr int TC_M = 128;
constexpr int TC_N = 2 * TC_MAX_NRHS;  // 64 accumulator columns
constexpr int TC_KC = 32;              // FP32 columns of A per chunk: one 128-byte swizzle row
constexpr int TC_BPS = 4;              // TMA boxes (sub-chunks) per stage
constexpr int TC_R = 2;                // stages in the ring
constexpr int TC_THREADS = 608;        // 19 warps: TMA (A), MMA, 8 split, 8 epilogue, TMA (B')
constexpr int TC_NA = 4;               // A operand buffers (TMEM, hi/lo)
constexpr int TC_NBB = 6;              // B' operand buffers (shared, hi/lo)
constexpr uint32_t TC_A_BYTES = TC_M * TC_KC * 4;  // 16 KB: one box, one sub-chunk
constexpr uint32_t TC_STAGE_BYTES = TC_BPS * TC_A_BYTES;
constexpr uint32_t TC_B_BYTES = TC_N * TC_KC * 4;  // 8 KB
constexpr uint32_t TC_BBUF = 2 * TC_B_BYTES;       // B' hi, lo
constexpr uint32_t TC_RING = TC_R * TC_STAGE_BYTES;
// TMEM: two accumulators of 128 columns (hi(A) hi(B') in 0-63, hi(A) lo(B') in
// 64-127) at columns 0 and 128, A operand buffers (hi 32 + lo 32 columns each) from 256
constexpr uint32_t TC_TMEM_COLS = 512;
constexpr uint32_t TC_ACC_COLS = 2 * TC_N;
constexpr uint32_t TC_ACC_COL = 0, TC_AOP_COL = 2 * TC_ACC_COLS;
static_assert(TC_AOP_COL + TC_NA * 64 <= TC_TMEM_COLS, "accumulators and operand buffers exceed the TMEM allocation");
constexpr int TC_NBARS = 2 * TC_R + 2 * TC_NA + 4 + 2 * TC_NBB;
constexpr size_t TC_SMEM = size_t(TC_RING) + TC_NBB * size_t(TC_BBUF) + 1024 + 256;
static_assert(8 * TC_NBARS + 4 <= 256, "barriers and the TMEM slot exceed their shared-memory space");
constexpr uint32_t TC_SPIN = 1u << 21;  // try_wait rounds before a wait is declared failed

static_assert(TC_BBUF % 1024 == 0 && TC_A_BYTES % 1024 == 0 && TC_B_BYTES % 1024 == 0, "swizzle atoms are 1 KB aligned");
static_assert(TC_SMEM <= 227 * 1024, "ring and operand buffers exceed the shared memory of a CTA");

// instruction descriptor, kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits
// 7-9, 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 at bits 17-22, M >> 4 at 24-28
constexpr uint32_t tc_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | (uint32_t(n >> 3) << 17) | (uint32_t(TC_M >> 4) << 24);
}
constexpr uint32_t TC_IDESC_N64 = tc_idesc(TC_N), TC_IDESC_N128 = tc_idesc(2 * TC_N);

// shared-memory matrix descriptor of a K-major operand in the 128-byte swizzled
// layout: start address >> 4 (bits 0-13), leading byte offset 16 B (unused for
// this layout, bits 16-29), stride byte offset 1024 B between 8-row groups
// (bits 32-45), descriptor version 1 (bit 46), swizzle mode 2 = 128 B (bits 61-63)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return uint64_t((saddr & 0x3FFFFu) >> 4) | (uint64_t(1) << 16) | (uint64_t(1024 >> 4) << 32) | (uint64_t(1) << 46) |
         (uint64_t(2) << 61);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// bounded wait for the phase of parity `parity` to complete; gives up early
// when another warp recorded a failure in *fail (shared memory)
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* fail = nullptr) {
  for (uint32_t it = 0; it < TC_SPIN; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
    if (fail && (it & 63) == 63 && *fail) return false;
  }
  return false;
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* map, int x, int y, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(bar)
      : "memory");
}
// D (TMEM) (+)= A (TMEM: lane = row, one TF32 per column) x B (shared memory descriptor)
__device__ __forceinline__ void tc_mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
      "r"(a_tmem), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 8 consecutive accumulator columns of this warp's 32 TMEM lanes, at two column offsets
__device__ __forceinline__ void tmem_ld8x2(uint32_t taddr, uint32_t off, float (&v)[8], float (&w)[8]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8, %9, %10, %11, %12, %13, %14, %15}, [%17];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr), "r"(taddr + off)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    v[i] = __uint_as_float(r[i]);
    w[i] = __uint_as_float(r[8 + i]);
  }
}
// 16 consecutive TMEM columns of this warp's 32 lanes from registers
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16};\n" ::"r"(taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

// FP32 -> TF32 (10 mantissa bits), round to nearest, ties away from zero: the
// result is an FP32 value with its 13 low mantissa bits zero, which the MMA
// takes exactly.  On the bit pattern: add half of the dropped unit (0x1000,
// carrying into the exponent when the mantissa overflows) and clear the 13
// bits - two full-rate integer operations (finite inputs below ~3.4e38)
__device__ __forceinline__ float tf32_rn(float v) {
  return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xFFFFE000u);
}
// v = hi + lo: hi = tf32(v) (|v - hi| <= 2^-11 |v|), lo = tf32(v - hi) (rounding
// error <= 2^-11 |v - hi| <= 2^-22 |v|), both exact TF32 operands
__device__ __forceinline__ void tf32_split(float v, float& hi, float& lo) {
  hi = tf32_rn(v);
  lo = tf32_rn(v - hi);
}


}  // namespace

// 19 warps over the 4 SM sub-partitions (5, 5, 5, 4) x 32 threads x 96 registers <= 16,384 each
__global__ void __maxnreg__(96)
    gemm_tc_kernel(const GemvJob* __restrict__ jobs, const unsigned char* __restrict__ maps, const TcTile* __restrict__ tiles,
                   const int32_t* __restrict__ cta_begin, const unsigned char* __restrict__ bmap,
                   const int32_t* __restrict__ job_base, int nrhs, int* err) {
  extern __shared__ unsigned char tc_raw[];
  const int t_begin = cta_begin[blockIdx.x], t_end = cta_begin[blockIdx.x + 1];
  if (t_begin >= t_end) return;
  const uint32_t raw = smem_u32(tc_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;  // ring[R], B'[NB]
  unsigned char* gb = tc_raw + (base - raw);
  const uint32_t bbuf0 = base + TC_RING;
  const uint32_t bars = bbuf0 + TC_NBB * TC_BBUF;
  // barriers (8 bytes each): full[R], empty[R], ready[NA], wfree[NA], accfull[2], accempty[2], bfull[NBB], bfree[NBB]
  auto full = [&](int s) { return bars + 8u * uint32_t(s); };
  auto empty = [&](int s) { return bars + 8u * uint32_t(TC_R + s); };
  auto ready = [&](int b) { return bars + 8u * uint32_t(2 * TC_R + b); };
  auto wfree = [&](int b) { return bars + 8u * uint32_t(2 * TC_R + TC_NA + b); };
  auto accfull = [&](int a) { return bars + 8u * uint32_t(2 * TC_R + 2 * TC_NA + a); };
  auto accempty = [&](int a) { return bars + 8u * uint32_t(2 * TC_R + 2 * TC_NA + 2 + a); };
  auto bfull = [&](int b) { return bars + 8u * uint32_t(2 * TC_R + 2 * TC_NA + 4 + b); };
  auto bfree = [&](int b) { return bars + 8u * uint32_t(2 * TC_R + 2 * TC_NA + 4 + TC_NBB + b); };
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(gb + (bars - base) + 8 * TC_NBARS);
  __shared__ int s_fail;
  volatile int* vfail = &s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

  if (tid == 0) {
    for (int q = 0; q < TC_R; ++q) {
      mbar_init(full(q), 1);
      mbar_init(empty(q), 8);
    }
    for (int b = 0; b < TC_NA; ++b) {
      mbar_init(ready(b), 8);
      mbar_init(wfree(b), 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(accfull(a), 1);
      mbar_init(accempty(a), 8);
    }
    for (int b = 0; b < TC_NBB; ++b) {
      mbar_init(bfull(b), 1);
      mbar_init(bfree(b), 1);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  // sub-chunks of a tile, padded to whole stages
  auto nk_of = [&](int t) { return tiles[t].nk; };
  int total = 0;  // sub-chunks of this CTA (a multiple of TC_BPS)
  for (int t = t_begin; t < t_end; ++t) total += nk_of(t);
  const int nstages = total / TC_BPS;

  if (warp == 0) {
    // ---------------- TMA producer: one stage = 4 boxes along K
    if (lane == 0) {
      int tile = t_begin, k = 0, nk = nk_of(t_begin), st = 0;
      for (; st < nstages; ++st) {
        const int q = st % TC_R;
        if (st >= TC_R && !mbar_wait(empty(q), uint32_t(((st / TC_R) - 1) & 1), vfail)) {
          *vfail = 1;
          break;
        }
        const TcTile T = tiles[tile];
        mbar_expect_tx(full(q), TC_STAGE_BYTES);
#pragma unroll
        for (int bx = 0; bx < TC_BPS; ++bx)
          tma_load_2d(base + uint32_t(q) * TC_STAGE_BYTES + uint32_t(bx) * TC_A_BYTES, maps + size_t(T.job) * 128,
                      (T.k0 + k + bx) * TC_KC, T.row0, full(q));
        k += TC_BPS;
        if (k == nk) {
          k = 0;
          if (++tile < t_end) nk = nk_of(tile);
        }
      }
      // the loads in flight (the latest stage of each slot) land before the CTA leaves
      for (int q = (st > TC_R ? st - TC_R : 0); q < st; ++q) mbar_wait(full(q % TC_R), uint32_t((q / TC_R) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int tile_i = 0, k = 0, nk = nk_of(t_begin), last = -1;
      for (int g = 0; g < total; ++g) {
        const int b = g % TC_NA, bb = g % TC_NBB, seg = g / TC_BPS, j = g % TC_BPS;
        bool ok = true;
        if (j == 0 && seg >= 2) ok = mbar_wait(accempty(seg & 1), uint32_t(((seg >> 1) - 1) & 1), vfail);
        if (ok) ok = mbar_wait(ready(b), uint32_t((g / TC_NA) & 1), vfail);
        if (ok) ok = mbar_wait(bfull(bb), uint32_t((g / TC_NBB) & 1), vfail);
        if (!ok) {
          *vfail = 1;
          break;
        }
        tc_fence_after();
        const uint32_t acc = tmem + TC_ACC_COL + uint32_t(seg & 1) * TC_ACC_COLS;
        const uint32_t aop = tmem + TC_AOP_COL + uint32_t(b) * 64u;  // hi at +0, lo at +32
        const uint32_t bh = bbuf0 + uint32_t(bb) * TC_BBUF;           // B' hi rows 0-63, lo rows 64-127
#pragma unroll
        for (int ks = 0; ks < TC_KC / 8; ++ks) {
          const uint32_t o = uint32_t(ks) * 32u;  // 8 TF32 = 32 bytes along K in the swizzle row of B'
          const uint32_t ac = uint32_t(ks) * 8u;  // 8 TMEM columns of A
          const uint32_t acc0 = (j > 0 || ks > 0) ? 1u : 0u;  // a fresh accumulator per segment
          // hi(A) [hi(B') | lo(B')] in one N = 128 product, then lo(A) hi(B') into columns 0-63
          tc_mma_ts(acc, aop + ac, sw128_desc(bh + o), TC_IDESC_N128, acc0);
          tc_mma_ts(acc, aop + 32u + ac, sw128_desc(bh + o), TC_IDESC_N64, 1u);
        }
        tc_commit(wfree(b));
        tc_commit(bfree(bb));
        if (j == TC_BPS - 1) tc_commit(accfull(seg & 1));
        last = g;
        if (++k == nk) {
          k = 0;
          ++tile_i;
          if (t_begin + tile_i < t_end) nk = nk_of(t_begin + tile_i);
        }
      }
      // the MMAs in flight (they complete in order) finish before the CTA leaves
      if (last >= 0) {
        mbar_wait(wfree(last % TC_NA), uint32_t((last / TC_NA) & 1));
        mbar_wait(bfree(last % TC_NBB), uint32_t((last / TC_NBB) & 1));
      }
    }
    __syncwarp();
  } else if (warp < 10) {
    // ---------------- split warps: thread = row of the tile (TMEM lane quarter warp % 4); the
    // two warps of a lane quarter take the K columns 16 kh .. 16 kh + 15 of each sub-chunk
    const int q4 = warp & 3, kh = (warp - 2) >> 2, row = 32 * q4 + lane;
    for (int g = 0; g < total; ++g) {
      const int st = g / TC_BPS, j = g % TC_BPS, q = st % TC_R, b = g % TC_NA;
      bool ok = mbar_wait(full(q), uint32_t((st / TC_R) & 1), vfail);
      if (ok && g >= TC_NA) ok = mbar_wait(wfree(b), uint32_t(((g / TC_NA) - 1) & 1), vfail);
      ok = __all_sync(0xffffffffu, ok);  // the TMEM stores below need the whole warp
      if (!ok) {
        *vfail = 1;
        break;
      }
      // this row's half of box j of the landed stage: 4 x 16 B, swizzled
      const unsigned char* rp = gb + size_t(q) * TC_STAGE_BYTES + size_t(j) * TC_A_BYTES + size_t(row) * 128;
      float h[16], l[16];
#pragma unroll
      for (int jj = 0; jj < 4; ++jj) {
        const float4 a = *reinterpret_cast<const float4*>(rp + (((4 * kh + jj) ^ (row & 7)) * 16));
        tf32_split(a.x, h[4 * jj], l[4 * jj]);
        tf32_split(a.y, h[4 * jj + 1], l[4 * jj + 1]);
        tf32_split(a.z, h[4 * jj + 2], l[4 * jj + 2]);
        tf32_split(a.w, h[4 * jj + 3], l[4 * jj + 3]);
      }
      const uint32_t ta = tmem + (uint32_t(32 * q4) << 16) + TC_AOP_COL + uint32_t(b) * 64u + uint32_t(16 * kh);
      tmem_st16(ta, h);
      tmem_st16(ta + 32u, l);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      tc_fence_before();
      __syncwarp();
      if (lane == 0) {
        if (j == TC_BPS - 1) mbar_arrive(empty(q));  // the stage's last sub-chunk: it may be refilled
        mbar_arrive(ready(b));                        // A of this sub-chunk is in TMEM
      }
    }
  } else if (warp == 18) {
    // ---------------- TMA producer of B' (hi rows 0-63, lo rows 64-127 of one box per
    // sub-chunk, built for the pass by tc_bprime_kernel) into the operand buffers
    if (lane == 0) {
      int tile = t_begin, k = 0, nk = nk_of(t_begin), g = 0;
      for (; g < total; ++g) {
        const int b = g % TC_NBB;
        if (g >= TC_NBB && !mbar_wait(bfree(b), uint32_t(((g / TC_NBB) - 1) & 1), vfail)) {
          *vfail = 1;
          break;
        }
        mbar_expect_tx(bfull(b), TC_BBUF);
        tma_load_2d(bbuf0 + uint32_t(b) * TC_BBUF, bmap, 0, 2 * TC_N * (job_base[tiles[tile].job] + tiles[tile].k0 + k),
                    bfull(b));
        if (++k == nk) {
          k = 0;
          if (++tile < t_end) nk = nk_of(tile);
        }
      }
      // the loads in flight land before the CTA leaves
      for (int q = (g > TC_NBB ? g - TC_NBB : 0); q < g; ++q) mbar_wait(bfull(q % TC_NBB), uint32_t((q / TC_NBB) & 1));
    }
    __syncwarp();
  } else {
    // ---------------- epilogue warps: TMEM lane quarter warp % 4, accumulator columns 32 half ..
    const int q4 = warp & 3, half = (warp - 10) >> 2;
    float cs[32], cc[32];  // compensated sums of this row's 32 columns over the tile's segments
#pragma unroll
    for (int i = 0; i < 32; ++i) cs[i] = cc[i] = 0.f;
    int seg = 0;
    for (int t = t_begin; t < t_end; ++t) {
      const int nseg = nk_of(t) / TC_BPS;
      bool ok = true;
      for (int sg = 0; sg < nseg; ++sg, ++seg) {
        ok = __all_sync(0xffffffffu, mbar_wait(accfull(seg & 1), uint32_t((seg >> 1) & 1), vfail));
        if (!ok) break;  // the TMEM loads below need the whole warp
        tc_fence_after();
#pragma unroll
        for (int hq = 0; hq < 4; ++hq) {
          float v[8], w[8];  // hi(A) hi(B') + lo(A) hi(B'), and hi(A) lo(B')
          tmem_ld8x2(tmem + (uint32_t(32 * q4) << 16) + TC_ACC_COL + uint32_t(seg & 1) * TC_ACC_COLS +
                         uint32_t(half * 32 + 8 * hq),
                     TC_N, v, w);
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = __fadd_rn(v[i], w[i]);
#pragma unroll
          for (int i = 0; i < 8; ++i) {  // TwoSum (Knuth): cs + cc carries the running sum
            const int c = 8 * hq + i;
            const float sum = __fadd_rn(cs[c], v[i]);
            const float bp = __fsub_rn(sum, cs[c]);
            cc[c] = __fadd_rn(cc[c], __fadd_rn(__fsub_rn(cs[c], __fsub_rn(sum, bp)), __fsub_rn(v[i], bp)));
            cs[c] = sum;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(accempty(seg & 1));  // the accumulator may take the next segment
      }
      if (!ok) {
        *vfail = 1;
        break;
      }
      const TcTile T = tiles[t];
      const GemvJob J = jobs[T.job];
      const int row = T.row0 + 32 * q4 + lane;
      if (row < J.m) {
        float2* y = reinterpret_cast<float2*>(J.y);
        const float ar = float(J.ar), ai = float(J.ai);
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int r = half * 16 + c;
          if (r < nrhs) {
            const float re = cs[2 * c] + cc[2 * c], im = cs[2 * c + 1] + cc[2 * c + 1];
            float2 o = make_float2(ar * re - ai * im, ar * im + ai * re);
            float2* yy = y + int64_t(r) * J.ldy + row;
            if (T.split) {
              atomicAdd(yy, o);  // one of the two K halves of the tile (Y zeroed before the pass)
            } else {
              if (J.beta) {
                const float2 bb = *yy;
                o.x += bb.x;
                o.y += bb.y;
              }
              *yy = o;
            }
          }
        }
      }
#pragma unroll
      for (int i = 0; i < 32; ++i) cs[i] = cc[i] = 0.f;
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && *vfail) atomicExch(err, 1);
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
}

// B' of every sub-chunk of the pass (hi rows 0-63, lo rows 64-127, 32 FP32 columns
// each, row-major; TMA applies the 128-byte swizzle): for right-hand side r and
// complex column c = 16 kc + u / 2 of the sub-chunk's job, row 2r holds
// (Re x_r[c], -Im x_r[c]) and row 2r + 1 (Im x_r[c], Re x_r[c]) at columns u, u + 1
// (u even), TF32 hi and lo parts; zero for r >= nrhs and beyond the job's columns.
// Blocks nsub and above zero the Y rows of the tiles split along K.
__global__ void tc_bprime_kernel(const GemvJob* __restrict__ jobs, const int32_t* __restrict__ gjob,
                                 const int32_t* __restrict__ gkc, int nsub, const TcTile* __restrict__ ztiles, int nrhs,
                                 float* __restrict__ bp) {
  const int gidx = blockIdx.x;
  if (gidx >= nsub) {  // Y rows of a tile split along K: zeroed, the two halves add into them
    const TcTile T = ztiles[gidx - nsub];
    const GemvJob& J = jobs[T.job];
    float2* y = reinterpret_cast<float2*>(J.y);
    for (int e = threadIdx.x; e < TC_M * nrhs; e += blockDim.x) {
      const int row = T.row0 + e % TC_M, r = e / TC_M;
      if (row < J.m) y[int64_t(r) * J.ldy + row] = make_float2(0.f, 0.f);
    }
    return;
  }
  const GemvJob& J = jobs[gjob[gidx]];
  const int kc = gkc[gidx];
  const float2* x = reinterpret_cast<const float2*>(J.x);
  for (int e = threadIdx.x; e < TC_N * TC_KC / 2; e += blockDim.x) {  // (row, complex column) pairs
    const int brow = e / (TC_KC / 2), cl = e % (TC_KC / 2);
    const int r = brow >> 1, c = kc * (TC_KC / 2) + cl;
    float2 v = make_float2(0.f, 0.f);
    if (r < nrhs && c < J.n) v = x[int64_t(r) * J.ldx + c];
    const float a0 = (brow & 1) ? v.y : v.x, a1 = (brow & 1) ? v.x : -v.y;
    float h0, l0, h1, l1;
    tf32_split(a0, h0, l0);
    tf32_split(a1, h1, l1);
    float* hi = bp + (size_t(gidx) * 2 * TC_N + brow) * TC_KC + 2 * cl;
    float* lo = hi + size_t(TC_N) * TC_KC;
    *reinterpret_cast<float2*>(hi) = make_float2(h0, h1);
    *reinterpret_cast<float2*>(lo) = make_float2(l0, l1);
  }
}

// ---------------------------------------------------------------- host side
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                                  const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encoder() {
  // looked up once (thread-safe initialisation of a local static)
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      return reinterpret_cast<EncodeTiledFn>(p);
    return EncodeTiledFn(nullptr);
  }();
  return fn;
}

void tc_plan_build(const std::vector<GemvJob>& jobs, TcPlan& tp, cudaStream_t s) {
  tp.ok = false;
  EncodeTiledFn enc = encoder();
  if (!enc || jobs.empty()) return;
  static_assert(sizeof(CUtensorMap) == 128, "tensor map size");
  std::vector<unsigned char> maps(jobs.size() * 128);
  std::vector<TcTile> tl;
  std::vector<int> cost;
  std::vector<int32_t> job_base, gjob, gkc;
  std::vector<TcTile> tp_zero;  // tiles split along K: their Y rows are zeroed before each pass
  for (size_t i = 0; i < jobs.size(); ++i) {
    const GemvJob& J = jobs[i];
    const uint64_t pitch = uint64_t(J.lda) * 8;
    if (J.m <= 0 || J.n <= 0 || pitch % 16 != 0 || (reinterpret_cast<uintptr_t>(J.A) & 15) != 0) return;
    alignas(64) CUtensorMap map;
    const cuuint64_t dims[2] = {cuuint64_t(2) * J.n, cuuint64_t(J.m)};
    const cuuint64_t strides[1] = {pitch};
    const cuuint32_t box[2] = {cuuint32_t(TC_KC), cuuint32_t(TC_M)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(J.A), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return;
    std::memcpy(&maps[i * 128], &map, 128);
    const int nk = ((2 * J.n + TC_KC - 1) / TC_KC + TC_BPS - 1) / TC_BPS * TC_BPS;
    job_base.push_back(int32_t(gjob.size()));
    for (int kc = 0; kc < nk; ++kc) {
      gjob.push_back(int32_t(i));
      gkc.push_back(kc);
    }
    for (int r0 = 0; r0 < J.m; r0 += TC_M) {
      tl.push_back({int32_t(i), r0, 0, nk, 0});
      cost.push_back(nk);
    }
  }
  int dev = 0, nsm = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  SLDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // Tiles are whole rows of 128 x the job's K: a few long tiles against the SM
  // count leave CTAs idle at the end (the longest-first assignment of 180 tiles
  // of one length to 152 CTAs gives 28 of them two).  Tiles longer than 0.3 of
  // a CTA's mean load are split into two K halves (whole stages) that add into
  // Y atomically: two additions into zero commute, so the result stays
  // independent of their order.  Jobs that accumulate into Y (beta) keep whole tiles.
  {
    long long tot = 0;
    for (int c : cost) tot += c;
    const double lim = 0.3 * double(tot) / double(std::max(1, std::min<int>(nsm, int(tl.size()))));
    const size_t n0 = tl.size();
    for (size_t i = 0; i < n0; ++i) {
      if (cost[i] < 4 * TC_BPS || double(cost[i]) <= lim || jobs[tl[i].job].beta) continue;
      const int h = cost[i] / TC_BPS / 2 * TC_BPS;
      TcTile b = tl[i];
      b.k0 = h;
      b.nk = cost[i] - h;
      b.split = 1;
      tl[i].nk = h;
      tl[i].split = 1;
      cost[i] = h;
      tp_zero.push_back(tl[i]);
      tl.push_back(b);
      cost.push_back(b.nk);
    }
  }
  // longest tiles first, each to the least loaded CTA
  const int nctas = std::max(1, std::min<int>(nsm, int(tl.size())));
  std::vector<size_t> order(tl.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
  std::vector<std::vector<TcTile>> per(nctas);
  typedef std::pair<long long, int> LoadCta;
  std::priority_queue<LoadCta, std::vector<LoadCta>, std::greater<LoadCta>> pq;
  for (int c = 0; c < nctas; ++c) pq.push({0, c});
  for (size_t i : order) {
    LoadCta lc = pq.top();
    pq.pop();
    per[lc.second].push_back(tl[i]);
    pq.push({lc.first + cost[i], lc.second});
  }
  std::vector<TcTile> flat;
  std::vector<int32_t> begin(1, 0);
  for (auto& v : per) {
    flat.insert(flat.end(), v.begin(), v.end());
    begin.push_back(int32_t(flat.size()));
  }
  // B' for every sub-chunk and its tensor map (boxes of 128 rows x 128 B, swizzled like the A boxes)
  tp.nsub = int(gjob.size());
  tp.bprime.alloc(size_t(tp.nsub) * 2 * TC_N * TC_KC);
  {
    alignas(64) CUtensorMap bm;
    const cuuint64_t dims[2] = {cuuint64_t(TC_KC), cuuint64_t(tp.nsub) * 2 * TC_N};
    const cuuint64_t strides[1] = {cuuint64_t(TC_KC) * 4};
    const cuuint32_t box[2] = {cuuint32_t(TC_KC), cuuint32_t(2 * TC_N)};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(&bm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, tp.bprime.p, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return;
    std::vector<unsigned char> bmv(128);
    std::memcpy(bmv.data(), &bm, 128);
    tp.bmap.upload(bmv, s);
  }
  tp.nzero = int(tp_zero.size());
  if (tp.nzero > 0) tp.ztiles.upload(tp_zero, s);
  tp.job_base.upload(job_base, s);
  tp.gjob.upload(gjob, s);
  tp.gkc.upload(gkc, s);
  tp.maps.upload(maps, s);
  tp.tiles.upload(flat, s);
  tp.cta_begin.upload(begin, s);
  tp.err.alloc(1);
  tp.err.zero(s);
  tp.nctas = nctas;
  SLDM_CUDA(cudaStreamSynchronize(s));
  tp.ok = true;
}

void gemm_tc(const GemvPlan& plan, const TcPlan& tp, int nrhs, cudaStream_t s) {
  SLDM_REQUIRE(tp.ok && nrhs >= 1 && nrhs <= TC_MAX_NRHS, SLDM_EINVAL, "tensor-core product: invalid plan or nrhs");
  static std::atomic<uint64_t> attr_set{0};  // devices whose attribute is set
  int dev = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(attr_set.load() & bit)) {
    SLDM_CUDA(cudaFuncSetAttribute(gemm_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(TC_SMEM)));
    attr_set.fetch_or(bit);
  }
  ScopedTimer tm("gemm_tc", s);
  tc_bprime_kernel<<<unsigned(tp.nsub + tp.nzero), 256, 0, s>>>(plan.jobs, tp.gjob.p, tp.gkc.p, tp.nsub, tp.ztiles.p, nrhs,
                                                                tp.bprime.p);
  count_launch();
  gemm_tc_kernel<<<unsigned(tp.nctas), TC_THREADS, TC_SMEM, s>>>(plan.jobs, tp.maps.p, tp.tiles.p, tp.cta_begin.p,
                                                                  tp.bmap.p, tp.job_base.p, nrhs, tp.err.p);
  count_launch();
  SLDM_CUDA(cudaGetLastError());
}

void tc_check(const TcPlan& tp, cudaStream_t s) {
  if (!tp.ok) return;
  int h = 0;
  SLDM_CUDA(cudaMemcpyAsync(&h, tp.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  if (h) {
    SLDM_CUDA(cudaMemsetAsync(tp.err.p, 0, sizeof(int), s));
    throw Error{SLDM_ETIMEOUT, "tensor-core product: a bounded wait ran out"};
  }
}

}  // namespace sldm
