// Y E by inner solves for large objects: FP32 approximate inverse of M_l and
// FP64 iterative refinement (see nested.h).
#include <cmath>
#include <complex>

#include "nested.h"

namespace sldm {

static __global__ void nested_c64_kernel(int64_t n, const double2* __restrict__ a, float2* __restrict__ b) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) b[i] = make_float2(float(a[i].x), float(a[i].y));
}

static __global__ void identity_kernel(int64_t n, float2* __restrict__ b) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n * n) b[i] = make_float2(i / n == i % n ? 1.f : 0.f, 0.f);
}

// wt1[e0 + i] = y[i] / ell (i < ne), wt2[q0 + i] = ell y[ne + i] (i < nq), per column
static __global__ void nested_out_kernel(int ne, int nq, int nr, const double2* __restrict__ y, int64_t ldw, double ell,
                                  double2* __restrict__ wt1, int64_t ld1, double2* __restrict__ wt2, int64_t ld2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (c >= nr || i >= ne + nq) return;
  const double2 v = y[int64_t(c) * ldw + i];
  if (i < ne) wt1[int64_t(c) * ld1 + i] = make_double2(v.x / ell, v.y / ell);
  else wt2[int64_t(c) * ld2 + (i - ne)] = make_double2(v.x * ell, v.y * ell);
}

// copy nr columns of n entries (column strides ld)
static __global__ void copy_cols_kernel(int64_t n, int nr, const double2* __restrict__ a, double2* __restrict__ b, int64_t ld) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int c = blockIdx.y;
  if (i < n && c < nr) b[int64_t(c) * ld + i] = a[int64_t(c) * ld + i];
}

// A plan of one GEMV job (the tiles of the several-right-hand-side kernel
// included), uploaded to the given buffers.
static void one_job_plan(const GemvJob& j, size_t es_m, size_t es_v, const char* name, DBuf<GemvJob>& dj,
                         DBuf<int64_t>& drs, DBuf<int2>& dt, GemvPlan& p) {
  std::vector<GemvJob> jobs{j};
  std::vector<int64_t> rs{0};
  std::vector<int2> tiles;
  for (int r0 = 0; r0 < j.m; r0 += gemv_tile_rows(es_v)) tiles.push_back(make_int2(0, r0));
  dj.upload(jobs);
  drs.upload(rs);
  dt.upload(tiles);
  p.name = name;
  p.jobs = dj.p;
  p.rowstart = drs.p;
  p.njobs = 1;
  p.total_rows = j.m;
  p.tiles = dt.p;
  p.ntiles = int(tiles.size());
  p.tile_rows = gemv_tile_rows(es_v);
  p.has_lo = false;
  p.bytes = double(j.m) * j.n * es_m;
  p.tc = nullptr;
}

static double host_norm(const std::vector<double2>& v) {
  double s = 0;
  for (const double2& a : v) s += a.x * a.x + a.y * a.y;
  return std::sqrt(s);
}

bool nested_setup(NestedMat& mat, cudaStream_t s) {
  const int64_t n = mat.n;
  {
    // X = M_l^-1 in complex64: the blocked LU of a complex64 copy with B = I
    DBuf<float2> A32;
    A32.alloc(size_t(n) * n);
    mat.X.alloc(size_t(n) * n);
    const int64_t nn = n * n;
    nested_c64_kernel<<<unsigned((nn + 255) / 256), 256, 0, s>>>(nn, mat.M.p, A32.p), count_launch();
    identity_kernel<<<unsigned((nn + 255) / 256), 256, 0, s>>>(n, mat.X.p), count_launch();
    SLDM_CUDA(cudaGetLastError());
    ScopedTimer tm("nested_inverse", s);
    lu_solve_batched<float2>({LUSysT<float2>{A32.p, mat.X.p, int32_t(n), int32_t(n)}}, s);
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  // the contraction on a test vector: e_i = exp(j i) / sqrt(ne), t = R e
  std::vector<double2> e(mat.ne);
  for (int i = 0; i < mat.ne; ++i) e[i] = make_double2(std::cos(double(i)), std::sin(double(i)));
  DBuf<double2> de, t, y, r;
  de.upload(e, s);
  t.alloc(n);
  y.alloc(n);
  r.alloc(n);
  DBuf<GemvJob> j1, j2, j3, j4;
  DBuf<int64_t> r1, r2, r3, r4;
  DBuf<int2> t1, t2, t3, t4;
  GemvPlan pR, pX0, pM, pXa;
  one_job_plan({mat.R.p, mat.ne, int32_t(n), mat.ne, de.p, mat.ne, t.p, n, 1, 0, 0, 0, nullptr}, 16, 16, "nested_R", j1, r1,
               t1, pR);
  one_job_plan({mat.X.p, n, int32_t(n), int32_t(n), t.p, n, y.p, n, 1, 0, 0, 0, nullptr}, 8, 16, "nested_X", j2, r2, t2, pX0);
  one_job_plan({mat.M.p, n, int32_t(n), int32_t(n), y.p, n, r.p, n, -1, 0, 1, 0, nullptr}, 16, 16, "nested_M", j3, r3, t3, pM);
  one_job_plan({mat.X.p, n, int32_t(n), int32_t(n), r.p, n, y.p, n, 1, 0, 1, 0, nullptr}, 8, 16, "nested_X", j4, r4, t4, pXa);
  gemv_jobs_mixed<double2, double2>(pR, 1, s);
  gemv_jobs_mixed<float2, double2>(pX0, 1, s);
  std::vector<double2> h(n);
  SLDM_CUDA(cudaMemcpyAsync(h.data(), t.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  const double tn = host_norm(h);
  if (!(tn > 0)) return false;
  double prev = tn;
  double worst = 0;
  for (int k = 1; k <= 12; ++k) {
    SLDM_CUDA(cudaMemcpyAsync(r.p, t.p, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    gemv_jobs_mixed<double2, double2>(pM, 1, s);  // r = t - M y
    SLDM_CUDA(cudaMemcpyAsync(h.data(), r.p, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
    SLDM_CUDA(cudaStreamSynchronize(s));
    const double rn = host_norm(h);
    if (!std::isfinite(rn)) return false;
    worst = std::max(worst, rn / prev);
    if (rn <= 1e-13 * tn) {
      mat.steps = k + 1;  // k - 1 corrections reached it: apply makes k (one for margin)
      mat.contraction = worst;
      return worst < 0.3;
    }
    if (rn > 0.3 * prev) return false;
    prev = rn;
    gemv_jobs_mixed<float2, double2>(pXa, 1, s);  // y += X r
  }
  return false;
}

void nested_plans(NestedUse& u, const double2* e, int64_t lde, double2* t, double2* y, double2* r, int64_t ldw) {
  NestedMat& m = *u.mat;
  const int64_t n = m.n;
  one_job_plan({m.R.p, m.ne, int32_t(n), m.ne, e + u.e0, lde, t, ldw, 1, 0, 0, 0, nullptr}, 16, 16, "nested_R", u.jR, u.rR,
               u.tR, u.pR);
  one_job_plan({m.X.p, n, int32_t(n), int32_t(n), t, ldw, y, ldw, 1, 0, 0, 0, nullptr}, 8, 16, "nested_X", u.jX0, u.rX0,
               u.tX0, u.pX0);
  one_job_plan({m.M.p, n, int32_t(n), int32_t(n), y, ldw, r, ldw, -1, 0, 1, 0, nullptr}, 16, 16, "nested_M", u.jM, u.rM, u.tM,
               u.pM);
  one_job_plan({m.X.p, n, int32_t(n), int32_t(n), r, ldw, y, ldw, 1, 0, 1, 0, nullptr}, 8, 16, "nested_X", u.jXa, u.rXa,
               u.tXa, u.pXa);
}

void nested_apply(const NestedUse& u, const double2* t, double2* y, double2* r, int64_t ldw, double2* wt1, int64_t ld1,
                  double2* wt2, int64_t ld2, int nr, double ell, cudaStream_t s) {
  const NestedMat& m = *u.mat;
  ScopedTimer tm("nested_y", s);
  gemv_jobs_mixed<double2, double2>(u.pR, nr, s);   // t = R e
  gemv_jobs_mixed<float2, double2>(u.pX0, nr, s);   // y = X t
  for (int k = 1; k < m.steps; ++k) {
    copy_cols_kernel<<<dim3(unsigned((m.n + 255) / 256), nr), 256, 0, s>>>(m.n, nr, t, r, ldw), count_launch();
    gemv_jobs_mixed<double2, double2>(u.pM, nr, s);  // r = t - M y
    gemv_jobs_mixed<float2, double2>(u.pXa, nr, s);  // y += X r
  }
  nested_out_kernel<<<dim3(unsigned((m.n + 127) / 128), nr), 128, 0, s>>>(m.ne, m.nq, nr, y, ldw, ell, wt1 + u.e0, ld1,
                                                                        wt2 + u.q0, ld2),
      count_launch();
  SLDM_CUDA(cudaGetLastError());
}

}  // namespace sldm
