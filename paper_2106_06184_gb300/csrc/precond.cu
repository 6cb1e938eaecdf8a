// Sparse block preconditioner P of Sec. III (Eq. pcext) and its analytic
// inverse through the Schur complement of the charge block:
//
//   P = [ diag L^A_m    diag I_x   D^T diag(L^phi_m) B       ]
//       [ diag mu L^A  -diag K     D^T diag(L^phi/eps) B     ]
//       [ F D           0          k0^2 I                    ]
//
// (row 2 carries -diag K, as the final system's row 2 carries -K).  With
// Lambda the per-edge inverse of the 2x2 block [[a, b], [c, d]] of diagonals,
// P x = r is solved by
//   S x3 = r3 - F D (L11 r1 + L12 r2),  S = k0^2 I - F D (L11 P13 + L12 P23),
//   [x1; x2] = Lambda ([r1; r2] - [P13; P23] x3).
// S is block diagonal by object (D, B, F are); each block is formed on the
// device and inverted once per assembly with the batched LU.
#include "dense.h"
#include "precond.h"

namespace sldm {

__device__ __forceinline__ double2 c_mul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
template <class C>
__device__ __forceinline__ double2 ld2(const C* p, int64_t i) { return make_double2(double(p[i].x), double(p[i].y)); }

// per edge: Lambda = [[a, b], [c, d]]^-1 with a = L^A_m[m,m], b = I_x[m,m], c = (mu L^A)[m,m], d = -K[m,m]
template <class C>
__global__ void prec_edges_kernel(int ne, const int32_t* __restrict__ tplus, const int32_t* __restrict__ tri_obj,
                                  const PrecObj* __restrict__ objs, const C* __restrict__ LAm, const char* __restrict__ loc,
                                  const int32_t* __restrict__ ix_ptr, const int32_t* __restrict__ ix_col,
                                  const double* __restrict__ ix_val, double2* lam) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ne) return;
  const PrecObj O = objs[tri_obj[tplus[m]]];
  const int ml = m - O.e0;
  const double2 a = ld2(LAm, int64_t(m) * ne + m);
  double bx = 0;
  for (int z = ix_ptr[m]; z < ix_ptr[m + 1]; ++z)
    if (ix_col[z] == m) bx = ix_val[z];
  const double2 b = make_double2(bx, 0.0);
  const C* LA = reinterpret_cast<const C*>(loc) + O.oLA;
  const C* K = reinterpret_cast<const C*>(loc) + O.oK;
  const double2 c = ld2(LA, int64_t(ml) * O.ne + ml);
  const double2 kd = ld2(K, int64_t(ml) * O.ne + ml);
  const double2 d = make_double2(-kd.x, -kd.y);
  const double2 det = c_sub(c_mul(a, d), c_mul(b, c));
  const double2 one = make_double2(1.0, 0.0);
  const double2 idet = c_div(one, det);
  lam[4 * m + 0] = c_mul(d, idet);
  lam[4 * m + 1] = c_mul(make_double2(-b.x, -b.y), idet);
  lam[4 * m + 2] = c_mul(make_double2(-c.x, -c.y), idet);
  lam[4 * m + 3] = c_mul(a, idet);
}

// per triangle: diagonals of L^phi_m (global) and of the object's L^phi/eps
template <class C>
__global__ void prec_tris_kernel(int nt, const int32_t* __restrict__ tri_obj, const PrecObj* __restrict__ objs,
                                 const C* __restrict__ LPm, const char* __restrict__ loc, double2* pdiag) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const PrecObj O = objs[tri_obj[t]];
  const int tl = t - O.t0;
  const C* LP = reinterpret_cast<const C*>(loc) + O.oLP;
  pdiag[2 * t + 0] = ld2(LPm, int64_t(t) * nt + t);
  pdiag[2 * t + 1] = ld2(LP, int64_t(tl) * O.nt + tl);
}

// S_o[q, q2] = k0^2 delta - sum_{edges e of t(q)} D[t(q), e] (L11[e] P13[e, q2] + L12[e] P23[e, q2])
// P13[e, q2] = D[t(q2), e] pm[t(q2)] - D[last, e] pm[last]  (P23 with the object's diagonal)
// Writes S_o (row-major) and the identity right-hand side for its inversion.
__global__ void prec_schur_kernel(const PrecObj O, double k0, const int32_t* __restrict__ tri_edge,
                                  const int8_t* __restrict__ tri_sign, const int32_t* __restrict__ tplus,
                                  const int32_t* __restrict__ tminus, const double2* __restrict__ lam,
                                  const double2* __restrict__ pdiag, double2* S, double2* I) {
  const int nq = O.nt - 1;
  const int q2 = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = blockIdx.y;
  if (q2 >= nq) return;
  const int t = O.t0 + q, t2 = O.t0 + q2, last = O.t0 + O.nt - 1;
  double2 acc = make_double2(q == q2 ? k0 * k0 : 0.0, 0.0);
  for (int i = 0; i < 3; ++i) {
    const int e = tri_edge[3 * t + i];
    const double s = double(tri_sign[3 * t + i]);  // D[t, e]
    const double d2 = (tplus[e] == t2) ? 1.0 : ((tminus[e] == t2) ? -1.0 : 0.0);
    const double dl = (tplus[e] == last) ? 1.0 : ((tminus[e] == last) ? -1.0 : 0.0);
    if (d2 == 0.0 && dl == 0.0) continue;
    const double2 p13 = c_sub(make_double2(d2 * pdiag[2 * t2].x, d2 * pdiag[2 * t2].y),
                              make_double2(dl * pdiag[2 * last].x, dl * pdiag[2 * last].y));
    const double2 p23 = c_sub(make_double2(d2 * pdiag[2 * t2 + 1].x, d2 * pdiag[2 * t2 + 1].y),
                              make_double2(dl * pdiag[2 * last + 1].x, dl * pdiag[2 * last + 1].y));
    const double2 v = c_add(c_mul(lam[4 * e + 0], p13), c_mul(lam[4 * e + 1], p23));
    acc.x -= s * v.x;
    acc.y -= s * v.y;
  }
  S[int64_t(q) * nq + q2] = acc;
  I[int64_t(q) * nq + q2] = make_double2(q == q2 ? 1.0 : 0.0, 0.0);
}

template <class CV>
__device__ __forceinline__ CV to_cv(double2 v);
template <>
__device__ __forceinline__ double2 to_cv<double2>(double2 v) { return v; }
template <>
__device__ __forceinline__ float2 to_cv<float2>(double2 v) { return make_float2(float(v.x), float(v.y)); }

// t3 = r3 - F D (L11 r1 + L12 r2) (per charge unknown; column blockIdx.y)
template <class CV>
__global__ void prec_apply1_kernel(int ne, int nq, const int32_t* __restrict__ q2t, const int32_t* __restrict__ tri_edge,
                                   const int8_t* __restrict__ tri_sign, const double2* __restrict__ lam,
                                   const double2* __restrict__ r, int64_t ld, CV* t3) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  r += int64_t(blockIdx.y) * ld;
  const int t = q2t[q];
  double2 acc = r[2 * ne + q];
  for (int i = 0; i < 3; ++i) {
    const int e = tri_edge[3 * t + i];
    const double s = double(tri_sign[3 * t + i]);
    const double2 v = c_add(c_mul(lam[4 * e + 0], r[e]), c_mul(lam[4 * e + 1], r[ne + e]));
    acc.x -= s * v.x;
    acc.y -= s * v.y;
  }
  t3[int64_t(blockIdx.y) * nq + q] = to_cv<CV>(acc);
}

// full charges bx = B x3 per object (the last triangle carries minus the sum),
// one CTA per object and column
template <class CV>
__global__ void prec_apply3_kernel(const PrecObj* __restrict__ objs, int nq_all, int nt, const CV* __restrict__ x3,
                                   double2* bx) {
  const PrecObj O = objs[blockIdx.x];
  x3 += int64_t(blockIdx.y) * nq_all;
  bx += int64_t(blockIdx.y) * nt;
  const int nq = O.nt - 1;
  double sr = 0, si = 0;
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const CV v = x3[O.q0 + q];
    bx[O.t0 + q] = make_double2(double(v.x), double(v.y));
    sr += double(v.x);
    si += double(v.y);
  }
  __shared__ double rr[256], ri[256];
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      rr[threadIdx.x] += rr[threadIdx.x + w];
      ri[threadIdx.x] += ri[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) bx[O.t0 + O.nt - 1] = make_double2(-rr[0], -ri[0]);
}

// x1, x2 = Lambda (r1 - P13 x3, r2 - P23 x3); x3 copied into the output (column blockIdx.y)
template <class CV>
__global__ void prec_apply45_kernel(int ne, int nq, int nt, const int32_t* __restrict__ tplus,
                                    const int32_t* __restrict__ tminus, const double2* __restrict__ lam,
                                    const double2* __restrict__ pdiag, const double2* __restrict__ r, int64_t ld,
                                    const double2* __restrict__ bx, const CV* __restrict__ x3, double2* x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  r += int64_t(blockIdx.y) * ld;
  x += int64_t(blockIdx.y) * ld;
  bx += int64_t(blockIdx.y) * nt;
  x3 += int64_t(blockIdx.y) * nq;
  if (i < ne) {
    const int tp = tplus[i], tm = tminus[i];
    const double2 y1 = c_sub(r[i], c_sub(c_mul(pdiag[2 * tp], bx[tp]), c_mul(pdiag[2 * tm], bx[tm])));
    const double2 y2 = c_sub(r[ne + i], c_sub(c_mul(pdiag[2 * tp + 1], bx[tp]), c_mul(pdiag[2 * tm + 1], bx[tm])));
    x[i] = c_add(c_mul(lam[4 * i + 0], y1), c_mul(lam[4 * i + 1], y2));
    x[ne + i] = c_add(c_mul(lam[4 * i + 2], y1), c_mul(lam[4 * i + 3], y2));
  }
  if (i < nq) x[2 * ne + i] = make_double2(double(x3[i].x), double(x3[i].y));
}

__global__ void to_c64_kernel(int64_t n, const double2* __restrict__ a, float2* b) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = make_float2(float(a[i].x), float(a[i].y));
}

template <class C>
void prec_setup(Precond& P, const sldm_mesh* m, const std::vector<PrecObj>& objs, double k0, const void* LAm,
                const void* LPm, const char* loc, const double* ix_val, cudaStream_t s) {
  const HostMesh& h = m->h;
  const DevMesh& d = m->d;
  const int ne = int(h.ne), nt = int(h.nt);
  P.objs.upload(objs, s);
  P.lam.alloc(size_t(4) * ne);
  P.pdiag.alloc(size_t(2) * nt);
  prec_edges_kernel<C><<<(ne + 127) / 128, 128, 0, s>>>(ne, d.tplus.p, d.obj.p, P.objs.p, (const C*)LAm, loc, d.ix_ptr.p,
                                                        d.ix_col.p, ix_val, P.lam.p), ::sldm::count_launch();
  prec_tris_kernel<C><<<(nt + 127) / 128, 128, 0, s>>>(nt, d.obj.p, P.objs.p, (const C*)LPm, loc, P.pdiag.p), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
  int64_t tot = 0;
  std::vector<int64_t> off;
  for (auto& o : objs) {
    off.push_back(tot);
    tot += int64_t(o.nt - 1) * (o.nt - 1);
  }
  DBuf<double2> Sm;
  Sm.alloc(tot);
  P.sinv.alloc(tot);
  std::vector<LUSys> sys;
  for (size_t i = 0; i < objs.size(); ++i) {
    const PrecObj& o = objs[i];
    const int nq = o.nt - 1;
    prec_schur_kernel<<<dim3((nq + 127) / 128, nq), 128, 0, s>>>(o, k0, d.tri_edge.p, d.tri_sign.p, d.tplus.p, d.tminus.p,
                                                                P.lam.p, P.pdiag.p, Sm.p + off[i], P.sinv.p + off[i]), ::sldm::count_launch();
    sys.push_back({Sm.p + off[i], P.sinv.p + off[i], nq, nq});
  }
  SLDM_CUDA(cudaGetLastError());
  lu_solve_batched(sys, s);  // sinv <- S^-1
  // a complex64 operator takes an FP32 preconditioner: S^-1 (inverted in FP64)
  // rounded to complex64, applied with FP32 arithmetic
  P.f32 = sizeof(C) == sizeof(float2);
  if (P.f32 && tot > 0) {
    P.sinv32.alloc(tot);
    to_c64_kernel<<<std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, s>>>(tot, P.sinv.p, P.sinv32.p), ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
    SLDM_CUDA(cudaStreamSynchronize(s));
    P.sinv.release();
  }
  // GEMV plan: x3_o = S_o^-1 t3_o, WR columns of nq
  const size_t ev = P.f32 ? sizeof(float2) : sizeof(double2);
  P.nq = h.nt - h.nobj;
  const int64_t nq1 = std::max<int64_t>(P.nq, 1);
  P.t3.alloc(nq1 * MAX_NRHS);
  P.x3.alloc(nq1 * MAX_NRHS);
  P.bx.alloc(h.nt * MAX_NRHS);
  std::vector<GemvJob> jobs;
  std::vector<int64_t> rs;
  std::vector<int2> tiles;
  int64_t acc = 0;
  const char* A0 = P.f32 ? (const char*)P.sinv32.p : (const char*)P.sinv.p;
  for (size_t i = 0; i < objs.size(); ++i) {
    const int nq = objs[i].nt - 1;
    if (nq <= 0) continue;
    for (int r0 = 0; r0 < nq; r0 += gemv_tile_rows(ev)) tiles.push_back(make_int2(int(jobs.size()), r0));
    jobs.push_back({A0 + off[i] * ev, nq, nq, nq, (char*)P.t3.p + objs[i].q0 * ev, P.nq, (char*)P.x3.p + objs[i].q0 * ev,
                    P.nq, 1, 0, 0, 0});
    rs.push_back(acc);
    acc += nq;
  }
  P.jobs.upload(jobs, s);
  P.rs.upload(rs, s);
  P.tiles.upload(tiles, s);
  P.plan.jobs = P.jobs.p;
  P.plan.rowstart = P.rs.p;
  P.plan.njobs = int(jobs.size());
  P.plan.total_rows = acc;
  P.plan.tiles = P.tiles.p;
  P.plan.ntiles = int(tiles.size());
  P.plan.tile_rows = gemv_tile_rows(ev);
  P.plan.name = "gemv_pc";
  P.plan.bytes = 0;
  for (auto& jb : jobs) P.plan.bytes += double(jb.m) * jb.n * ev;
  P.plan.tc = nullptr;
  if (P.f32) {
    tc_plan_build(jobs, P.tc, s);
    if (P.tc.ok) P.plan.tc = &P.tc;
  }
  SLDM_CUDA(cudaStreamSynchronize(s));
}

template <class CV>
static void prec_apply_t(const Precond& P, const sldm_mesh* m, const double2* r, double2* x, int64_t ld, int nr,
                         cudaStream_t s) {
  const HostMesh& h = m->h;
  const DevMesh& d = m->d;
  const int ne = int(h.ne), nq = int(P.nq), nt = int(h.nt);
  CV* t3 = reinterpret_cast<CV*>(P.t3.p);
  CV* x3 = reinterpret_cast<CV*>(P.x3.p);
  if (nq > 0) {
    prec_apply1_kernel<CV><<<dim3((nq + 255) / 256, nr), 256, 0, s>>>(ne, nq, d.q2t.p, d.tri_edge.p, d.tri_sign.p, P.lam.p,
                                                                       r, ld, t3), ::sldm::count_launch();
    gemv_jobs<CV>(P.plan, nr, s);
  }
  prec_apply3_kernel<CV><<<dim3(unsigned(h.nobj), nr), 256, 0, s>>>(P.objs.p, nq, nt, x3, P.bx.p), ::sldm::count_launch();
  const int n = std::max(ne, nq);
  prec_apply45_kernel<CV><<<dim3((n + 255) / 256, nr), 256, 0, s>>>(ne, nq, nt, d.tplus.p, d.tminus.p, P.lam.p, P.pdiag.p,
                                                                     r, ld, P.bx.p, x3, x), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

void prec_apply(const Precond& P, const sldm_mesh* m, const double2* r, double2* x, int64_t ld, int nr, cudaStream_t s) {
  ScopedTimer tm("precond", s);
  SLDM_REQUIRE((nr >= 1 && nr <= MAX_NRHS), SLDM_EINVAL, "preconditioner: 1 to 32 columns");
  if (P.f32) prec_apply_t<float2>(P, m, r, x, ld, nr, s);
  else prec_apply_t<double2>(P, m, r, x, ld, nr, s);
}

template void prec_setup<float2>(Precond&, const sldm_mesh*, const std::vector<PrecObj>&, double, const void*, const void*,
                                 const char*, const double*, cudaStream_t);
template void prec_setup<double2>(Precond&, const sldm_mesh*, const std::vector<PrecObj>&, double, const void*, const void*,
                                  const char*, const double*, cudaStream_t);

}  // namespace sldm
