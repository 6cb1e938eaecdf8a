// Preconditioner P of Eq. pcext (precond.cu).
#pragma once
#include "dense.h"
#include "gemm_tc.h"

namespace sldm {

// Object description for the preconditioner (offsets are elements of the op's local block storage).
struct PrecObj {
  int32_t e0, ne, t0, nt, q0, pad;
  int64_t oLA, oK, oLP;
};

struct Precond {
  DBuf<PrecObj> objs;
  DBuf<double2> lam;    // 4 per edge: Lambda11, Lambda12, Lambda21, Lambda22
  DBuf<double2> pdiag;  // 2 per triangle: diag L^phi_m, diag of the object's L^phi/eps
  DBuf<double2> sinv;   // per object (nt_o - 1)^2: S_o^-1, row-major (complex128 operators)
  DBuf<float2> sinv32;  // the same in complex64 (complex64 operators: an FP32 preconditioner)
  bool f32 = false;
  // WR columns each: t3, x3 of nq (entries of the preconditioner's precision), bx of nt
  DBuf<double2> t3, x3, bx;
  int64_t nq = 0;
  DBuf<GemvJob> jobs;
  DBuf<int64_t> rs;
  DBuf<int2> tiles;
  GemvPlan plan;
  TcPlan tc;  // complex64: the Schur-inverse products on the tensor cores (9 to 32 columns)
  bool ready = false;
};

template <class C>
void prec_setup(Precond& P, const sldm_mesh* m, const std::vector<PrecObj>& objs, double k0, const void* LAm,
                const void* LPm, const char* loc, const double* ix_val, cudaStream_t s);
// x = P^-1 r for nr <= WR columns (complex128 vectors of length N, column stride ld)
void prec_apply(const Precond& P, const sldm_mesh* m, const double2* r, double2* x, int64_t ld, int nr, cudaStream_t s);

}  // namespace sldm
