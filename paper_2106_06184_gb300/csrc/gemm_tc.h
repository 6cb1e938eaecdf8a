// Multi-right-hand-side complex64 block products on the 5th-generation tensor
// cores (gemm_tc.cu): Y = alpha A X (+ Y) for 9 to 32 right-hand sides per pass.
#pragma once
#include "dense.h"

namespace sldm {

// Right-hand sides one tensor-core pass takes (accumulator width 2 x 32 FP32 columns).
constexpr int TC_MAX_NRHS = 32;

// 128 rows of a job from row0, over K sub-chunks [k0, k0 + nk) of 32 FP32
// columns (whole stages); split: one of two K halves of the rows, added into Y
struct TcTile {
  int32_t job, row0, k0, nk, split;
};

// Per GEMV plan: one TMA tensor map per job (the block seen as a row-major FP32
// matrix of m rows and 2n columns), the 128-row tiles of every job (long ones in
// two K halves), and their assignment to CTAs (longest first, to the least loaded CTA); the real-form
// right-hand-side operand B' of every K chunk, rebuilt for each pass.
struct TcPlan {
  DBuf<unsigned char> maps;  // 128-byte tensor maps, 64-byte aligned
  DBuf<TcTile> tiles;
  DBuf<int32_t> cta_begin;   // CTA c takes tiles [cta_begin[c], cta_begin[c + 1])
  DBuf<int> err;             // set to 1 by a CTA whose bounded wait ran out
  // B' of the pass (built from the vectors before each pass): sub-chunk g of the
  // plan is (job gjob[g], K chunk gkc[g]), job j's first sub-chunk job_base[j];
  // 128 rows x 32 FP32 per sub-chunk (hi, lo), read by TMA through bmap
  DBuf<float> bprime;
  DBuf<unsigned char> bmap;
  DBuf<int32_t> job_base, gjob, gkc;
  DBuf<TcTile> ztiles;       // the first halves of the split tiles (their Y rows are zeroed per pass)
  int nsub = 0, nzero = 0;
  int nctas = 0;
  bool ok = false;           // every job fits the tensor-core path
};

// Builds tp for the jobs of a complex64 plan (host copies of the jobs).  tp.ok is
// false (and the plan keeps the CUDA-core kernels) when a job's row pitch is
// not a multiple of 16 bytes or the driver's tensor-map encoder is unavailable.
void tc_plan_build(const std::vector<GemvJob>& jobs, TcPlan& tp, cudaStream_t s);
// One pass over every job of `plan` for nrhs (<= 32) right-hand sides.
void gemm_tc(const GemvPlan& plan, const TcPlan& tp, int nrhs, cudaStream_t s);
// SLDM_ETIMEOUT when a tensor-core pass recorded a bounded wait that ran out (reads and clears the flag).
void tc_check(const TcPlan& tp, cudaStream_t s);

}  // namespace sldm
