// Y E by inner solves for large objects (nested.cu).
//
// Sec. III of the paper forms Y = M_l^-1 R_l by direct factorisation only for
// objects below about a thousand triangles and solves M_l y = R_l e inside each
// product of the outer system otherwise.  Here the inner solve is iterative
// refinement in FP64 with an FP32 approximate inverse of the length-scaled M_l:
// X ~ M_l^-1 from the blocked LU in complex64 (A X = I), then
//   t = R_l e;  y = X t;  repeat `steps` times:  r = t - M_l y (FP64);  y += X r
// which contracts the error by ||I - M_l X|| per step.  `steps` is measured once
// at assembly on a test vector (the count that reaches 1e-13 of ||t||, plus one),
// so an application needs no host synchronisation.  When the contraction is too
// slow (ill-conditioned M_l) the caller keeps the FP64 LU instead.
#pragma once

#include <memory>
#include <vector>

#include "dense.h"

namespace sldm {

// The object's matrices (shared by the objects that repeat it).
struct NestedMat {
  int32_t n = 0, ne = 0, nq = 0;  // order of M_l, edges, triangles - 1
  DBuf<double2> M, R;              // row-major, length-scaled: M_l (n x n), R_l (n x ne)
  DBuf<float2> X;                  // complex64 approximation of M_l^-1 (n x n)
  int steps = 0;                   // refinement steps of every application
  double contraction = 0;          // measured ||r_{k+1}|| / ||r_k|| at assembly
};

// One object's use of a NestedMat: its slices of the structured product's work
// vectors and the GEMV plans that read and write them.
struct NestedUse {
  int obj = 0, mat_owner = 0;  // this object, the object whose M_l it shares
  std::shared_ptr<NestedMat> mat;
  int64_t e0 = 0, q0 = 0;
  DBuf<GemvJob> jR, jX0, jXa, jM;
  DBuf<int64_t> rR, rX0, rXa, rM;
  DBuf<int2> tR, tX0, tXa, tM;
  GemvPlan pR, pX0, pXa, pM;
};

// Builds X from mat.M and measures mat.steps; false when refinement would not
// reach 1e-13 within 12 steps (the caller then factors M_l in FP64).
bool nested_setup(NestedMat& mat, cudaStream_t s);

// Plans of object use u against the work vectors: e (edges, column stride lde),
// wt1 (edges, stride ld1), wt2 (triangles - objects, stride ld2) and the scratch
// t, y, r (n x WR complex128 each, column stride ldw).
void nested_plans(NestedUse& u, const double2* e, int64_t lde, double2* t, double2* y, double2* r, int64_t ldw);

// wt1 = Y11 e / ell and wt2 = ell Y21 e of object use u for nr columns (ell: the
// length scaling of M_l), by the refinement above.
void nested_apply(const NestedUse& u, const double2* t, double2* y, double2* r, int64_t ldw, double2* wt1, int64_t ld1,
                  double2* wt2, int64_t ld2, int nr, double ell, cudaStream_t s);

}  // namespace sldm
