// Declarations of the dense-algebra kernels (dense.cu).
#pragma once
#include "internal.h"

namespace sldm {

// One dense system A X = B solved in place (A: n x n, B: n x nrhs, row-major complex64 or complex128).
template <class C>
struct LUSysT {
  C* A;
  C* B;
  int32_t n, nrhs;
};
typedef LUSysT<double2> LUSys;
template <class C>
void lu_solve_batched(const std::vector<LUSysT<C>>& systems, cudaStream_t s);
// Blocked LU of one large system (lu_blocked.cu); lu_solve_batched sends there
// every system of order LU_BLOCKED_MIN or more (below that the look-ahead
// kernel, whose steps need no grid barrier, is faster).
constexpr int LU_BLOCKED_MIN = 1024;
template <class C>
void lu_solve_blocked(const LUSysT<C>& S, cudaStream_t s);
inline void lu_solve_batched(const std::vector<LUSys>& systems, cudaStream_t s) { lu_solve_batched<double2>(systems, s); }

template <class C>
void build_Ml(const sldm_mesh* m, int obj, double k0, const void* LAm, int64_t ldLA, const void* LPm, int64_t ldLP,
              const void* Kl, int64_t ldK, const double* ix_val, C* Ml, C* Rl, cudaStream_t s);

// y = (ar + j ai) A x + beta y over rows [0, m) of a row-major block; x, y hold
// nrhs columns with strides ldx, ldy (entries of the op precision).
struct GemvJob {
  const void* A;
  int64_t lda;
  int32_t m, n;
  const void* x;
  int64_t ldx;
  void* y;
  int64_t ldy;
  double ar, ai;
  int32_t beta, pad;
  // low parts of a complex64 block whose FP64 value is A + Alo (same layout and
  // lda), or null; read only by the FP64-accumulated complex64 product
  const void* Alo;
};
struct TcPlan;
// right-hand sides in lockstep (GMRES) and per pass of the structured product
// and the preconditioner: up to 32 (tensor cores for complex64 operators; the
// CUDA-core kernels take 8 per launch)
constexpr int MAX_NRHS = 32;
constexpr int TILE_NRHS = 8;
struct GemvPlan {
  const char* name = "gemv";   // timer name of its launches
  GemvJob* jobs = nullptr;     // device
  int64_t* rowstart = nullptr; // device, exclusive prefix sum of m
  int njobs = 0;
  int64_t total_rows = 0;
  // tiles of tile_rows rows of one job each (job, first row), device; used
  // with several right-hand sides (null: the one-row-per-warp kernel throughout)
  int2* tiles = nullptr;
  int ntiles = 0;
  int tile_rows = 0;
  // every job carries Alo (complex64 blocks with complex128 vectors only): the
  // product is that of the FP64 operator A + Alo
  bool has_lo = false;
  double bytes = 0;  // matrix bytes one launch streams (its timer's algorithmic units)
  // complex64 blocks and vectors: the tensor-core plan for 9 to 32 right-hand
  // sides per pass (gemm_tc.h), or null / not ok for passes of 8 on the CUDA cores
  const TcPlan* tc = nullptr;
  // smallest lockstep width sent to the tensor cores (set by gemv_autotune;
  // 33 = never): below it, passes of 8 on the CUDA cores
  int tc_from = TILE_NRHS + 1;
};
// right-hand sides in lockstep (GMRES) and per pass of the structured product
// and the preconditioner: up to 32 (tensor cores for complex64 operators; the
// CUDA-core kernels take 8 per launch)

// rows per tile of the several-right-hand-side kernel for vectors of es_v bytes
inline int gemv_tile_rows(size_t es_v) { return es_v == 8 ? 32 : 16; }
template <class C>
void gemv_jobs(const GemvPlan& plan, int nrhs, cudaStream_t s);
// complex64 matrix, complex128 vectors, FP64 accumulation
template <class CM, class CV>
void gemv_jobs_mixed(const GemvPlan& plan, int nrhs, cudaStream_t s);
// Measures, on this plan's own blocks, one complex64 pass at 16 and at 32
// right-hand sides on the tensor cores and as passes of 8 on the CUDA cores, and
// sets plan.tc_from to where the tensor cores start to win (9, 17 or 33 =
// never).  The plan's output vectors are overwritten; its inputs must hold
// finite values (the caller zeroes them).
void gemv_autotune(GemvPlan& plan, cudaStream_t s);

struct ApplyDims {
  int32_t ne, nt, nq, nobj;
};
template <class C>
void apply_glue_split(const double2* x, int64_t ldx, const ApplyDims& D, void* j, void* e, void* u, int nrhs, cudaStream_t s);
template <class C>
void apply_glue_prep(const sldm_mesh* m, const ApplyDims& D, const void* j, const void* u, const void* t1, const void* t2,
                     void* a, void* c, void* bc, void* bu, int nrhs, cudaStream_t s, const int32_t* tri_begin_dev,
                     const int32_t* edge_begin_dev);
template <class C>
void apply_glue_combine(const sldm_mesh* m, const ApplyDims& D, double k0, const double* ix_val, const void* z1,
                        const void* z2, const void* w1, const void* w2, const void* w3, const void* e, const void* a,
                        const void* c, double2* y, int64_t ldy, int nrhs, cudaStream_t s);

// One Gram-Schmidt pass over the Krylov bases of the live right-hand sides of a
// lockstep step: column k of each basis against its columns 0..k-1.  The
// bases have column stride ldv (a multiple of 64) and zero rows n..ldv-1.
struct KrylovStep {
  int64_t n = 0, ldv = 0;
  int k = 0, na = 0;
  void* V[MAX_NRHS] = {};       // basis of right-hand side j (complex64 or complex128)
  double2* h[MAX_NRHS] = {};    // its k projection coefficients (accumulated; cleared by the caller)
  double* nrm = nullptr;        // na squared norms of column k after an update with norm (cleared by the caller)
};
template <class CB>
void krylov_dots(const KrylovStep& ks, cudaStream_t s);                // h_j += V_j[:, :k]^H V_j[:, k]
template <class CB>
void krylov_update(const KrylovStep& ks, bool norm, cudaStream_t s);   // V_j[:, k] -= V_j[:, :k] h_j
template <class CX, class CY>
struct VecBatch {
  const CX* x[MAX_NRHS] = {};
  CY* y[MAX_NRHS] = {};
  double a[MAX_NRHS] = {};
};
// y_j = a_j s(i) x_j (s = s1 on [0, ne), s2 on [ne, 2 ne), s3 beyond), j < na, in place allowed
template <class CX, class CY>
void vscale3_batch(int64_t n, int64_t ne, double s1, double s2, double s3, const VecBatch<CX, CY>& b, int na,
                   cudaStream_t s);

// complex128 or complex64 storage (instantiated for double2 and float2; mixed
// pairs for vmul, vaxpby and vscale3)
template <class CB, class CW>
void vmul(const CB* V, int64_t ldv, int k, const double2* h, double sign, CW* w, int64_t n, cudaStream_t s);
template <class C>
void vnorm2(const C* w, int64_t n, double* out, cudaStream_t s);
template <class CX, class CY>
void vaxpby(int64_t n, double alpha, const CX* x, double beta, CY* y, cudaStream_t s);
template <class CX, class CY>
void vscale3(int64_t n, int64_t ne, double s1, double s2, double s3, const CX* x, CY* y, cudaStream_t s);

template <class C>
void to_c128(const void* src, int64_t n, double2* dst, cudaStream_t s);
// hi = complex64 rounding of src, lo = complex64 rounding of src - hi (src = hi + lo to ~2^-48)
void split_c128(const double2* src, int64_t n, float2* hi, float2* lo, cudaStream_t s);
// dst += lo (complex64 low parts onto a complex128 copy of the high parts)
void add_lo_c128(const float2* lo, int64_t n, double2* dst, cudaStream_t s);
template <class C>
void from_c128(const double2* src, int64_t n, void* dst, cudaStream_t s);
template <class C>
void copy_scaled(const void* src, int64_t n, double alpha, void* dst, cudaStream_t s);
// Copies of sub-blocks within one row-major matrix (leading dimension ld):
// rows [sr, sr + nr) x cols [sc, sc + nc) to [dr, dr + nr) x [dc, dc + nc).
// Sources are never destinations of the same call.
struct BlockCopy {
  int32_t sr, sc, dr, dc, nr, nc;
};
void copy_blocks(const std::vector<BlockCopy>& copies, size_t esz, void* M, int64_t ld, cudaStream_t s);
template <class C>
void add_ix(const sldm_mesh* m, int obj, double alpha, const double* ix_val, void* K, int64_t ld, cudaStream_t s);

// ---------------------------------------------------------------- GMRES on the device
// Per right-hand side r of a lockstep GMRES cycle: iterations, columns in use,
// whether it still iterates, ||b|| and the cycle's starting residual.
struct GmresState {
  int32_t it, kused, live, pad;
  double bnorm, beta;
};
// Step k of the Arnoldi process for the na active right-hand sides on[j]:
// column k of H_r from the two Gram-Schmidt passes (dh + r * ldh: coefficients
// of pass one at [0, k], pass two at [m + 2, m + 2 + k]) and h_{k+1,k} =
// sqrt(nrm[j]); the earlier Givens rotations, a new one annihilating h_{k+1,k},
// the rotated residual vector g_r; then the convergence tests (|g_{k+1}| <=
// tol ||b||, it >= maxit, h_{k+1,k} = 0, and with refine |g_{k+1}| <= cycle
// beta) clear live.  scale[j] = 1 / h_{k+1,k} for the next basis vector (0 once
// the right-hand side has stopped).  H: (m + 1) x m row-major per right-hand
// side, cs, sn: m, g: m + 1 (complex).
struct GivensArgs {
  int k, m, na, refine;
  const int* on;
  const double2* dh;
  int64_t ldh;
  const double* nrm;
  double2 *H, *cs, *sn, *g;
  GmresState* st;
  double tol, cycle;
  int maxit, pad;
  double* scale;
};
void gmres_givens(const GivensArgs& a, cudaStream_t s);
// y_r = H_r^-1 g_r (upper triangular, kused_r columns) into dh + r * ldh, for the na
// right-hand sides on[j] (one warp each).
void gmres_backsolve(int na, const int* on, int m, const double2* H, const double2* g, const GmresState* st, double2* dh,
                     int64_t ldh, cudaStream_t s);
// y_j = scale[j] x_j (scale on the device), j < na, in place allowed
template <class CB>
void vscale_dev_batch(int64_t n, const VecBatch<CB, CB>& b, const double* scale, int na, cudaStream_t s);

}  // namespace sldm
