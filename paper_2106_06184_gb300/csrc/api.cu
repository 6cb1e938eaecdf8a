// C ABI of libsldm (include/sldm.h): handle management, assembly of the
// single-layer dual-mesh operator (Sec. II-B to II-E), its structured product
// and the GMRES solver (Sec. IV).
#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <array>

#include "dense.h"
#include "gemm_tc.h"
#include "internal.h"
#include "mgf.h"
#include "nested.h"
#include "precond.h"

namespace sldm {

static thread_local std::string g_err;
void set_error(const std::string& m) { g_err = m; }

constexpr double PI_ = 3.14159265358979323846;
constexpr double C0_ = 299792458.0;
constexpr double MU0_ = 4e-7 * PI_;
constexpr double EPS0_ = 1.0 / (MU0_ * C0_ * C0_);

typedef std::complex<double> cplx;

struct ObjInfo {
  int32_t e0, ne, t0, nt, q0, nq;
  int64_t oLA, oLP, oK, oY11, oY21;  // element offsets in op->loc
  cplx k, eps_c;
  double mu_r;
  bool nested = false;  // Y E by inner solves (nested.h); Y11, Y21 are not formed
};

// Pinned flag buffers and events of the GMRES convergence polls (one per slot).
struct PollRing {
  static constexpr int SLOTS = 2;  // the host runs at most one step ahead of what it knows
  cudaEvent_t ev[SLOTS] = {};
  int32_t* flags[SLOTS] = {};
  bool ready = false;
  void init(int n) {
    if (ready) return;
    for (int i = 0; i < SLOTS; ++i) {
      SLDM_CUDA(cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming));
      SLDM_CUDA(cudaMallocHost(&flags[i], sizeof(int32_t) * n));
    }
    ready = true;
  }
  ~PollRing() {
    if (!ready) return;
    for (int i = 0; i < SLOTS; ++i) {
      cudaEventDestroy(ev[i]);
      cudaFreeHost(flags[i]);
    }
  }
};

}  // namespace sldm

struct sldm_op {
  const sldm_mesh* mesh = nullptr;
  int prec = SLDM_PREC_F64;   // storage of the solver's operator: SLDM_PREC_F64 or SLDM_PREC_F32
  bool x2 = false;            // SLDM_PREC_F32X2: complex64 operator plus the low parts of an FP64 fill
  size_t esz = 16;
  double k0 = 0, freq = 0;
  int device = 0;
  int64_t N = 0, ne = 0, nt = 0, nq = 0, nobj = 0;
  sldm::cplx kb, eps_b;
  double mu_b = 1;
  sldm::DBuf<char> LAm, LPm, loc;
  sldm::DBuf<char> LAm_lo, LPm_lo, loc_lo;  // SLDM_PREC_F32X2: FP64 value - complex64 value, in complex64
  std::vector<sldm::ObjInfo> obj;
  sldm::DBuf<double> ix_val;
  // structured product: work vectors for up to WR right-hand sides per pass
  static constexpr int WR = sldm::MAX_NRHS;
  sldm::DBuf<char> wj, we, wu, wt1, wt2, wa, wc, wbc, wbu, wz1, wz2, ww1, ww2, ww3;
  sldm::DBuf<sldm::GemvJob> jobs1, jobs2;
  sldm::DBuf<int64_t> rs1, rs2;
  sldm::DBuf<int2> tl1, tl2;
  sldm::GemvPlan plan1, plan2;
  sldm::TcPlan tc1, tc2;  // complex64: the same plans on the tensor cores (9 to 32 right-hand sides per pass)
  // complex64 operator applied with complex128 vectors (FP64 residuals of iterative refinement)
  sldm::DBuf<sldm::GemvJob> jobs1d, jobs2d;
  sldm::DBuf<int64_t> rs1d, rs2d;
  sldm::DBuf<int2> tl1d, tl2d;
  sldm::GemvPlan plan1d, plan2d;
  // layered background (external problem with the multilayer kernel)
  bool layered = false;
  sldm::MgfStackHost H;
  sldm::MgfTables T;
  std::vector<double> thick;
  double z_top = 0;
  // preconditioner of Eq. pcext
  sldm::Precond pc;
  // GMRES workspace
  int ws_m = 0;
  int64_t ldv = 0;  // column stride of the Krylov bases: N rounded up to 64, zero rows beyond N
  sldm::DBuf<double2> V, wb, wx, wr, wtmp, wtmp2, wacc, wz, dh;
  int ws_nr = 0;
  sldm::DBuf<double> dnorm;
  // GMRES on the device: Hessenberg, rotations, residual vectors, per right-hand side state
  sldm::DBuf<double2> gH, gcs, gsn, gg;
  sldm::DBuf<sldm::GmresState> gst;
  sldm::DBuf<double> gscale;
  sldm::DBuf<int> gon;
  sldm::PollRing polls;
  // large objects: Y E by inner solves (nested.h), and their scratch (n_max x WR)
  int nested_min = 2500;  // order of M_l from which Y is not formed (< 0: never)
  bool want_x2 = false;   // assembling for SLDM_PREC_F32X2 (split after the FP64 fill)
  std::vector<std::unique_ptr<sldm::NestedUse>> nested;
  sldm::DBuf<double2> wnt, wny, wnr;
  int64_t ldn = 0;
  std::mutex busy;
};

namespace sldm {

static int64_t op_bytes(const sldm_op* op) {
  int64_t nb = int64_t(op->wnt.bytes() + op->wny.bytes() + op->wnr.bytes());
  for (const auto& u : op->nested)
    if (u->mat && u->obj == u->mat_owner) nb += int64_t(u->mat->M.bytes() + u->mat->R.bytes() + u->mat->X.bytes());
  return nb + int64_t(op->LAm.bytes() + op->LPm.bytes() + op->loc.bytes() + op->LAm_lo.bytes() + op->LPm_lo.bytes() +
                 op->loc_lo.bytes() + op->ix_val.bytes() + op->V.bytes() +
                 op->pc.sinv.bytes() + op->pc.sinv32.bytes() + op->pc.lam.bytes() + op->pc.pdiag.bytes());
}

// GEMV plans of the structured product with matrix entries of es_m bytes and
// vector entries of es_v bytes (the work vectors hold complex128, so both the
// operator's precision and FP64 fit).
static void make_plans(sldm_op* op, size_t es_m, size_t es_v, DBuf<GemvJob>& dj1, DBuf<int64_t>& drs1, DBuf<int2>& dt1,
                       GemvPlan& p1, DBuf<GemvJob>& dj2, DBuf<int64_t>& drs2, DBuf<int2>& dt2, GemvPlan& p2,
                       TcPlan* tc1 = nullptr, TcPlan* tc2 = nullptr) {
  const int64_t ne = op->ne, nt = op->nt, nq = op->nq;
  auto P = [&](DBuf<char>& b, int64_t off) { return (void*)(b.p + off * es_v); };
  const char* loc = op->loc.p;
  auto L = [&](int64_t off) { return (const void*)(loc + off * es_m); };
  // the low parts (SLDM_PREC_F32X2) enter only the FP64-accumulated products
  const bool lo = op->x2 && es_v == sizeof(double2);
  auto Lo = [&](int64_t off) { return lo ? (const void*)(op->loc_lo.p + off * es_m) : nullptr; };
  const void* LAlo = lo ? op->LAm_lo.p : nullptr;
  const void* LPlo = lo ? op->LPm_lo.p : nullptr;
  std::vector<GemvJob> j1, j2;
  for (auto& o : op->obj) {
    if (o.nested) continue;  // Y E by inner solves in apply_dev
    j1.push_back({L(o.oY11), o.ne, o.ne, o.ne, P(op->we, o.e0), ne, P(op->wt1, o.e0), ne, 1, 0, 0, 0, Lo(o.oY11)});
    if (o.nq > 0)
      j1.push_back({L(o.oY21), o.ne, o.nq, o.ne, P(op->we, o.e0), ne, P(op->wt2, o.q0), nq, 1, 0, 0, 0, Lo(o.oY21)});
  }
  j2.push_back({op->LAm.p, ne, int32_t(ne), int32_t(ne), P(op->wa, 0), ne, P(op->wz1, 0), ne, 1, 0, 0, 0, LAlo});
  j2.push_back({op->LPm.p, nt, int32_t(nt), int32_t(nt), P(op->wbc, 0), nt, P(op->wz2, 0), nt, 1, 0, 0, 0, LPlo});
  for (auto& o : op->obj) {
    j2.push_back({L(o.oLA), o.ne, o.ne, o.ne, P(op->wj, o.e0), ne, P(op->ww1, o.e0), ne, 1, 0, 0, 0, Lo(o.oLA)});
    j2.push_back({L(o.oK), o.ne, o.ne, o.ne, P(op->we, o.e0), ne, P(op->ww2, o.e0), ne, 1, 0, 0, 0, Lo(o.oK)});
    j2.push_back({L(o.oLP), o.nt, o.nt, o.nt, P(op->wbu, o.t0), nt, P(op->ww3, o.t0), nt, 1, 0, 0, 0, Lo(o.oLP)});
  }
  auto mk = [&](std::vector<GemvJob>& j, DBuf<GemvJob>& dj, DBuf<int64_t>& drs, DBuf<int2>& dt, GemvPlan& plan,
                TcPlan* tc) {
    std::vector<int64_t> rs(j.size());
    std::vector<int2> tiles;
    int64_t acc = 0;
    for (size_t i = 0; i < j.size(); ++i) {
      rs[i] = acc;
      acc += j[i].m;
      for (int r0 = 0; r0 < j[i].m; r0 += gemv_tile_rows(es_v)) tiles.push_back(make_int2(int(i), r0));
    }
    dj.upload(j);
    drs.upload(rs);
    dt.upload(tiles);
    plan.jobs = dj.p;
    plan.rowstart = drs.p;
    plan.njobs = int(j.size());
    plan.total_rows = acc;
    plan.tiles = dt.p;
    plan.ntiles = int(tiles.size());
    plan.tile_rows = gemv_tile_rows(es_v);
    plan.has_lo = lo;
    plan.bytes = 0;
    for (auto& jb : j) plan.bytes += double(jb.m) * jb.n * es_m * (lo ? 2 : 1);
    plan.tc = nullptr;
    if (tc) {  // complex64 blocks and vectors: tensor-core passes of 9 to 32 right-hand sides
      tc_plan_build(j, *tc, 0);
      if (tc->ok) plan.tc = tc;
    }
  };
  mk(j1, dj1, drs1, dt1, p1, tc1);
  mk(j2, dj2, drs2, dt2, p2, tc2);
  p1.name = "gemv_y";     // Y11, Y21 (per object)
  p2.name = "gemv_main";  // L^A_m, L^phi_m and the internal blocks
}

template <class C>
static void build_plans(sldm_op* op, cudaStream_t s) {
  const int64_t ne = op->ne, nt = op->nt, nq = op->nq;
  const int WR = sldm_op::WR;
  const size_t ev = sizeof(double2);
  op->wj.alloc(ne * WR * ev); op->we.alloc(ne * WR * ev); op->wu.alloc(std::max<int64_t>(nq, 1) * WR * ev);
  op->wt1.alloc(ne * WR * ev); op->wt2.alloc(std::max<int64_t>(nq, 1) * WR * ev);
  op->wa.alloc(ne * WR * ev); op->wc.alloc(std::max<int64_t>(nq, 1) * WR * ev);
  op->wbc.alloc(nt * WR * ev); op->wbu.alloc(nt * WR * ev);
  op->wz1.alloc(ne * WR * ev); op->wz2.alloc(nt * WR * ev);
  op->ww1.alloc(ne * WR * ev); op->ww2.alloc(ne * WR * ev); op->ww3.alloc(nt * WR * ev);
  const bool c64 = sizeof(C) == sizeof(float2);
  make_plans(op, sizeof(C), sizeof(C), op->jobs1, op->rs1, op->tl1, op->plan1, op->jobs2, op->rs2, op->tl2, op->plan2,
             c64 ? &op->tc1 : nullptr, c64 ? &op->tc2 : nullptr);
  if (c64) {
    // where the tensor cores start to beat passes of 8 on the CUDA cores, measured
    // on this operator's own blocks (finite inputs: the work vectors zeroed)
    for (DBuf<char>* w : {&op->wj, &op->we, &op->wu, &op->wt1, &op->wt2, &op->wa, &op->wc, &op->wbc, &op->wbu, &op->wz1,
                          &op->wz2, &op->ww1, &op->ww2, &op->ww3})
      w->zero(s);
    gemv_autotune(op->plan1, s);
    gemv_autotune(op->plan2, s);
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  if (sizeof(C) == sizeof(float2)) {
    make_plans(op, sizeof(C), sizeof(double2), op->jobs1d, op->rs1d, op->tl1d, op->plan1d, op->jobs2d, op->rs2d, op->tl2d,
               op->plan2d);
    op->plan1d.name = "gemv_y_f64acc";
    op->plan2d.name = "gemv_main_f64acc";
  }
  if (!op->nested.empty()) {  // inner-solve objects: scratch of the largest M_l, and their plans
    int64_t nmax = 0;
    for (auto& u : op->nested) nmax = std::max<int64_t>(nmax, u->mat->n);
    op->ldn = (nmax + 63) / 64 * 64;
    op->wnt.alloc(size_t(op->ldn) * WR);
    op->wny.alloc(size_t(op->ldn) * WR);
    op->wnr.alloc(size_t(op->ldn) * WR);
    for (auto& u : op->nested)
      nested_plans(*u, reinterpret_cast<const double2*>(op->we.p), ne, op->wnt.p, op->wny.p, op->wnr.p, op->ldn);
  }
}

// y = Z x for nrhs columns, x/y complex128 on the device (column stride N)
// y = Z x: matrix entries CM, vectors and accumulation CV
template <class CM, class CV>
static void apply_dev(const sldm_op* op_, const double2* x, double2* y, int nrhs, cudaStream_t s, const GemvPlan& p1,
                      const GemvPlan& p2) {
  sldm_op* op = const_cast<sldm_op*>(op_);
  ApplyDims D{int32_t(op->ne), int32_t(op->nt), int32_t(op->nq), int32_t(op->nobj)};
  for (int r0 = 0; r0 < nrhs; r0 += sldm_op::WR) {
    int nr = std::min(sldm_op::WR, nrhs - r0);
    const double2* xr = x + int64_t(r0) * op->N;
    double2* yr = y + int64_t(r0) * op->N;
    apply_glue_split<CV>(xr, op->N, D, op->wj.p, op->we.p, op->wu.p, nr, s);
    if (p1.njobs > 0) gemv_jobs_mixed<CM, CV>(p1, nr, s);
    if (!op->nested.empty()) {
      if (sizeof(CV) != sizeof(double2)) throw Error{SLDM_EINVAL, "apply: inner-solve objects need complex128 vectors"};
      for (const auto& u : op->nested)
        nested_apply(*u, op->wnt.p, op->wny.p, op->wnr.p, op->ldn, reinterpret_cast<double2*>(op->wt1.p), op->ne,
                     reinterpret_cast<double2*>(op->wt2.p), op->nq, nr, op->mesh->h.ell, s);
    }
    apply_glue_prep<CV>(op->mesh, D, op->wj.p, op->wu.p, op->wt1.p, op->wt2.p, op->wa.p, op->wc.p, op->wbc.p, op->wbu.p, nr,
                        s, op->mesh->d.tri_begin.p, op->mesh->d.edge_begin.p);
    gemv_jobs_mixed<CM, CV>(p2, nr, s);
    apply_glue_combine<CV>(op->mesh, D, op->k0, op->ix_val.p, op->wz1.p, op->wz2.p, op->ww1.p, op->ww2.p, op->ww3.p,
                           op->we.p, op->wa.p, op->wc.p, yr, op->N, nr, s);
  }
}

// acc64: a complex64 operator's product with complex128 vectors, accumulated to
// ~48 bits (compensated FP32 sums of exactly split products; iterative refinement)
static void apply_any(const sldm_op* op, const double2* x, double2* y, int nrhs, cudaStream_t s, bool acc64 = false) {
  ScopedTimer tm("apply", s);
  if (op->prec == SLDM_PREC_F32) {
    if (acc64) apply_dev<float2, double2>(op, x, y, nrhs, s, op->plan1d, op->plan2d);
    else apply_dev<float2, float2>(op, x, y, nrhs, s, op->plan1, op->plan2);
  } else {
    apply_dev<double2, double2>(op, x, y, nrhs, s, op->plan1, op->plan2);
  }
}

static cplx eps_complex(double eps_r, double sigma, double omega) { return cplx(eps_r, -sigma / (omega * EPS0_)); }

// Objects o and r have the same shape when they have the same triangles and
// edges in the same local order (vertex and edge ids shifted by constants, the
// same edge signs) and vertices that differ by one translation to 1e-12 of the
// object's size; `shift` receives that translation (o's vertices minus r's).
static bool same_shape(const HostMesh& h, int o, int r, double shift[3]) {
  const int t0 = h.tri_begin[o], nt = h.tri_begin[o + 1] - t0, e0 = h.edge_begin[o], ne = h.edge_begin[o + 1] - e0;
  const int u0 = h.tri_begin[r], ue0 = h.edge_begin[r];
  if (h.tri_begin[r + 1] - u0 != nt || h.edge_begin[r + 1] - ue0 != ne) return false;
  if (h.bedge_begin[o + 1] - h.bedge_begin[o] != h.bedge_begin[r + 1] - h.bedge_begin[r]) return false;
  const int64_t dv = int64_t(h.tri[3 * size_t(t0)]) - h.tri[3 * size_t(u0)];
  double lo = 1e300, hi = -1e300;
  for (int d = 0; d < 3; ++d)
    shift[d] = h.xyz[3 * size_t(h.tri[3 * size_t(t0)]) + d] - h.xyz[3 * size_t(h.tri[3 * size_t(u0)]) + d];
  for (int i = 0; i < 3 * nt; ++i) {
    const size_t io = 3 * size_t(t0) + i, ir = 3 * size_t(u0) + i;
    if (!(int64_t(h.tri[io]) - h.tri[ir] == dv && h.tri_edge[io] - e0 == h.tri_edge[ir] - ue0 &&
          h.tri_sign[io] == h.tri_sign[ir]))
      return false;
  }
  for (int j = 0; j < ne; ++j)
    if (!(h.uv[2 * size_t(e0 + j)] - h.uv[2 * size_t(ue0 + j)] == dv &&
          h.uv[2 * size_t(e0 + j) + 1] - h.uv[2 * size_t(ue0 + j) + 1] == dv))
      return false;
  double dmax = 0;
  for (int i = 0; i < 3 * nt; ++i) {
    const size_t vo = size_t(h.tri[3 * size_t(t0) + i]), vr = size_t(h.tri[3 * size_t(u0) + i]);
    for (int d = 0; d < 3; ++d) {
      dmax = std::max(dmax, std::fabs(h.xyz[3 * vo + d] - h.xyz[3 * vr + d] - shift[d]));
      lo = std::min(lo, h.xyz[3 * vr + d]);
      hi = std::max(hi, h.xyz[3 * vr + d]);
    }
  }
  return dmax <= 1e-12 * (hi - lo);
}

// ref[o] = the first object that object o repeats, else o.  Object o repeats r
// when they have the same shape (same_shape) and the same material.  Interior
// blocks and Y depend only on that shape and material (the equivalent
// configuration uses the homogeneous kernel of the background layer, which a
// translation leaves unchanged), so they are filled once.
static std::vector<int> repeated_objects(const HostMesh& h, const sldm_material* mats) {
  const int nobj = int(h.nobj);
  std::vector<int> ref(nobj);
  double sh[3];
  for (int o = 0; o < nobj; ++o) {
    ref[o] = o;
    for (int r = 0; r < o && ref[o] == o; ++r) {
      if (ref[r] != r) continue;
      const sldm_material &a = mats[o], &b = mats[r];
      if (a.eps_r != b.eps_r || a.mu_r != b.mu_r || a.sigma != b.sigma || a.layer != b.layer) continue;
      if (same_shape(h, o, r, sh)) ref[o] = r;
    }
  }
  return ref;
}

// Reuse of the global blocks L^A_m, L^phi_m.  The block of object pair (i, j)
// (rows: i's edges or triangles, columns: j's) integrates G(r, r') over i's test
// and j's source triangles.  In a homogeneous background G depends on r - r'
// only, so two pairs whose objects have the same shapes at the same relative
// displacement have equal blocks; in a layered background G depends on the
// horizontal part of r - r' and on z and z' apart, so the pairs must also share
// the objects' heights.  `reps` lists one pair per distinct block (filled), the
// copies send each representative block to its repeats.  Objects of one shape
// class and their translations: cls[o], shift[o] (from the class's first object).
struct GlobalReuse {
  std::vector<std::pair<int, int>> reps;
  std::vector<BlockCopy> copyA, copyP;
};
static GlobalReuse global_reuse(const HostMesh& h, bool layered) {
  const int nobj = int(h.nobj);
  std::vector<int> cls(nobj);
  std::vector<std::array<double, 3>> shift(nobj);
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < h.nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], h.xyz[3 * v + d]);
      hi[d] = std::max(hi[d], h.xyz[3 * v + d]);
    }
  const double tol = 1e-12 * std::max({hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]});
  for (int o = 0; o < nobj; ++o) {
    cls[o] = o;
    shift[o] = {0.0, 0.0, 0.0};
    for (int r = 0; r < o; ++r) {
      if (cls[r] != r) continue;
      double sh[3];
      if (same_shape(h, o, r, sh)) {
        cls[o] = r;
        shift[o] = {sh[0], sh[1], sh[2]};
        break;
      }
    }
  }
  GlobalReuse g;
  struct Rep {
    int i, j;
    double d[3], zi;
  };
  std::map<std::pair<int, int>, std::vector<Rep>> by_cls;
  for (int i = 0; i < nobj; ++i)
    for (int j = 0; j < nobj; ++j) {
      double d[3];
      for (int k = 0; k < 3; ++k) d[k] = shift[j][k] - shift[i][k];
      const double zi = layered ? shift[i][2] : 0.0;
      auto& list = by_cls[{cls[i], cls[j]}];
      const Rep* hit = nullptr;
      for (const Rep& r : list)
        if (std::fabs(r.d[0] - d[0]) <= tol && std::fabs(r.d[1] - d[1]) <= tol && std::fabs(r.d[2] - d[2]) <= tol &&
            std::fabs(r.zi - zi) <= tol) {
          hit = &r;
          break;
        }
      if (!hit) {
        list.push_back({i, j, {d[0], d[1], d[2]}, zi});
        g.reps.push_back({i, j});
        continue;
      }
      const int ri = hit->i, rj = hit->j;
      g.copyA.push_back({h.edge_begin[ri], h.edge_begin[rj], h.edge_begin[i], h.edge_begin[j],
                         h.edge_begin[i + 1] - h.edge_begin[i], h.edge_begin[j + 1] - h.edge_begin[j]});
      g.copyP.push_back({h.tri_begin[ri], h.tri_begin[rj], h.tri_begin[i], h.tri_begin[j],
                         h.tri_begin[i + 1] - h.tri_begin[i], h.tri_begin[j + 1] - h.tri_begin[j]});
    }
  return g;
}

// Sommerfeld remainder tables of the objects' layer over the objects' extent:
// 256 log-spaced rho from 1e-3 of the shortest edge to 1.01 x the mesh diagonal,
// 128 points in z + z' and in |z - z'| over the objects' heights.
static void layered_tables(sldm_op* op, cudaStream_t s) {
  const HostMesh& h = op->mesh->h;
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int64_t v = 0; v < h.nv; ++v)
    for (int d = 0; d < 3; ++d) {
      lo[d] = std::min(lo[d], h.xyz[3 * v + d]);
      hi[d] = std::max(hi[d], h.xyz[3 * v + d]);
    }
  double span = 0, emin = 1e300;
  for (int d = 0; d < 3; ++d) span += (hi[d] - lo[d]) * (hi[d] - lo[d]);
  span = std::sqrt(span) * 1.01;
  for (int64_t n = 0; n < h.ne; ++n) {
    const double* p = &h.xyz[3 * h.uv[2 * n]];
    const double* q = &h.xyz[3 * h.uv[2 * n + 1]];
    emin = std::min(emin, std::sqrt((p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) + (p[2] - q[2]) * (p[2] - q[2])));
  }
  op->T.Q = mgf_static(op->H);
  mgf_build_tables(op->H, 2 * PI_ * op->freq, 1e-3 * emin, span, lo[2], hi[2], op->T, s);
}

template <class R>
static void assemble_impl(sldm_op* op, const sldm_material* mats, cudaStream_t s, bool finish = true) {
  typedef typename std::conditional<sizeof(R) == 4, float2, double2>::type C;
  const sldm_mesh* m = op->mesh;
  const HostMesh& h = m->h;
  const size_t es = sizeof(C);
  const double omega = 2 * PI_ * op->freq;
  // ---- external (global) blocks with the background wavenumber
  op->LAm.alloc(op->ne * op->ne * es);
  op->LPm.alloc(op->nt * op->nt * es);
  op->LAm.zero(s);
  op->LPm.zero(s);
  GlobalReuse gr;
  std::vector<RTask> rtasks;  // blocks of L^A_m, L^phi_m filled here (the rest are copies)
  {
    LTask t{};
    t.t0 = 0; t.ntest = int32_t(op->nt); t.s0 = 0; t.nsrc = int32_t(op->nt);
    t.ldA = op->ne; t.ldP = op->nt;
    t.A = op->LAm.p; t.P = op->LPm.p;
    t.kr = op->kb.real(); t.ki = op->kb.imag();
    t.sAr = op->mu_b; t.sAi = 0;
    cplx ip = 1.0 / op->eps_b;
    t.sPr = ip.real(); t.sPi = ip.imag();
    // repeated object pairs (arrays of identical objects) fill one block per
    // distinct relative placement; a background that splits sources (a good
    // conductor) keeps the single task, whose far-pair cut spans the whole fill
    if (op->nobj > 1 && !split_rules_L(h, t).split) gr = global_reuse(h, op->layered);
    if (!gr.copyA.empty()) {
      std::vector<LTask> tasks;
      for (auto& pr : gr.reps) {
        LTask u = t;
        u.t0 = h.tri_begin[pr.first];
        u.ntest = h.tri_begin[pr.first + 1] - u.t0;
        u.s0 = h.tri_begin[pr.second];
        u.nsrc = h.tri_begin[pr.second + 1] - u.s0;
        tasks.push_back(u);
        rtasks.push_back({u.t0, u.ntest, u.s0, u.nsrc});
      }
      fill_L<R>(m, tasks, s);
      // in a stack the repeats are copied once the reflected part is in
      if (!op->layered) {
        copy_blocks(gr.copyA, es, op->LAm.p, op->ne, s);
        copy_blocks(gr.copyP, es, op->LPm.p, op->nt, s);
      }
    } else {
      fill_L<R>(m, {t}, s);
      rtasks.push_back({0, int32_t(op->nt), 0, int32_t(op->nt)});
    }
  }
  // ---- per-object layout of the local blocks
  int64_t off = 0;
  op->obj.clear();
  for (int o = 0; o < op->nobj; ++o) {
    ObjInfo oi{};
    oi.e0 = h.edge_begin[o]; oi.ne = h.edge_begin[o + 1] - oi.e0;
    oi.t0 = h.tri_begin[o]; oi.nt = h.tri_begin[o + 1] - oi.t0;
    oi.q0 = oi.t0 - o; oi.nq = oi.nt - 1;
    oi.eps_c = eps_complex(mats[o].eps_r, mats[o].sigma, omega);
    oi.mu_r = mats[o].mu_r;
    oi.k = op->k0 * std::sqrt(oi.eps_c * oi.mu_r);
    auto al = [&](int64_t n) { int64_t r = off; off += (n + 1) & ~int64_t(1); return r; };  // keep 16-byte alignment
    oi.oLA = al(int64_t(oi.ne) * oi.ne);
    oi.oLP = al(int64_t(oi.nt) * oi.nt);
    oi.oK = al(int64_t(oi.ne) * oi.ne);
    oi.oY11 = al(int64_t(oi.ne) * oi.ne);
    oi.oY21 = al(int64_t(oi.nq) * oi.ne);
    op->obj.push_back(oi);
  }
  op->loc.alloc(off * es);
  op->loc.zero(s);
  char* loc = op->loc.p;
  // ---- objects that repeat an earlier one take its interior blocks and Y
  const std::vector<int> ref = repeated_objects(h, mats);
  // ---- internal L^A, L^phi with each object's wavenumber
  {
    std::vector<LTask> tasks;
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] != o) continue;
      const ObjInfo& oi = op->obj[o];
      LTask t{};
      t.t0 = oi.t0; t.ntest = oi.nt; t.s0 = oi.t0; t.nsrc = oi.nt;
      t.e_row0 = oi.e0; t.e_col0 = oi.e0; t.t_row0 = oi.t0; t.t_col0 = oi.t0;
      t.ldA = oi.ne; t.ldP = oi.nt;
      t.A = loc + oi.oLA * es; t.P = loc + oi.oLP * es;
      t.kr = oi.k.real(); t.ki = oi.k.imag();
      t.sAr = oi.mu_r; t.sAi = 0;
      cplx ip = 1.0 / oi.eps_c;
      t.sPr = ip.real(); t.sPi = ip.imag();
      tasks.push_back(t);
    }
    fill_L<R>(m, tasks, s);
  }
  // ---- Gram matrix I_x
  op->ix_val.alloc(std::max<size_t>(h.ix_col.size(), 1));
  gram_ix(m, op->ix_val.p, s);
  // ---- Kbar with BC sources: internal (k) and equivalent (k_l) per object
  int64_t kb_total = 0, kl_total = 0, ml_total = 0, rl_total = 0;
  std::vector<int64_t> kb_off, kl_off, ml_off, rl_off;
  for (int o = 0; o < op->nobj; ++o) {
    const ObjInfo& oi = op->obj[o];
    int64_t nbe = h.bedge_begin[o + 1] - h.bedge_begin[o];
    kb_off.push_back(kb_total); kb_total += int64_t(oi.ne) * nbe;
    kl_off.push_back(kl_total); kl_total += int64_t(oi.ne) * oi.ne;
    int64_t n = oi.ne + oi.nq;
    ml_off.push_back(ml_total); ml_total += n * n;
    rl_off.push_back(rl_total); rl_total += n * oi.ne;
  }
  DBuf<char> Kb, Kl;
  Kb.alloc(kb_total * es);
  Kl.alloc(kl_total * es);
  for (int pass = 0; pass < 2; ++pass) {
    Kb.zero(s);
    std::vector<KTask> tasks;
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] != o) continue;
      const ObjInfo& oi = op->obj[o];
      KTask t{};
      t.t0 = oi.t0; t.ntest = oi.nt; t.c0 = 6 * oi.t0; t.nsrc = 6 * oi.nt;
      t.e_row0 = oi.e0; t.b_col0 = h.bedge_begin[o];
      t.ld = h.bedge_begin[o + 1] - h.bedge_begin[o];
      t.Kb = Kb.p + kb_off[o] * es;
      cplx k = pass == 0 ? oi.k : op->kb;
      t.kr = k.real(); t.ki = k.imag();
      tasks.push_back(t);
    }
    fill_K<R>(m, tasks, s);
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] != o) continue;
      const ObjInfo& oi = op->obj[o];
      int64_t ld = h.bedge_begin[o + 1] - h.bedge_begin[o];
      void* dst = pass == 0 ? (void*)(loc + oi.oK * es) : (void*)(Kl.p + kl_off[o] * es);
      contract_bc<R>(m, o, Kb.p + kb_off[o] * es, ld, dst, oi.ne, s);
      if (pass == 0) add_ix<C>(m, o, 0.5, op->ix_val.p, dst, oi.ne, s);
    }
  }
  Kb.release();
  // ---- Y11, Y21 by LU of M_l, in the operator's precision (M_l uses the homogeneous
  //      kernel of the background layer: LAm/LPm hold only that part at this point)
  {
    DBuf<C> Ml, Rl;
    Ml.alloc(ml_total);
    Rl.alloc(rl_total);
    std::vector<LUSysT<C>> sys;
    // large objects of an FP64 operator: Y E by inner solves (nested.h) instead of Y
    auto inner = [&](const ObjInfo& oi) {
      return sizeof(C) == sizeof(double2) && !op->want_x2 && op->nested_min >= 0 && oi.ne + oi.nq >= op->nested_min;
    };
    std::vector<int> cand;
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] != o) continue;
      const ObjInfo& oi = op->obj[o];
      build_Ml<C>(m, o, op->k0, op->LAm.p, op->ne, op->LPm.p, op->nt, Kl.p + kl_off[o] * es, oi.ne, op->ix_val.p,
                  Ml.p + ml_off[o], Rl.p + rl_off[o], s);
      if (inner(oi)) cand.push_back(o);
      else sys.push_back({Ml.p + ml_off[o], Rl.p + rl_off[o], oi.ne + oi.nq, oi.ne});
    }
    lu_solve_batched<C>(sys, s);
    std::vector<std::shared_ptr<NestedMat>> nmat(op->nobj);
    if constexpr (sizeof(C) == sizeof(double2)) {
      std::vector<LUSysT<C>> fallback;  // refinement too slow: the FP64 LU after all
      for (int o : cand) {
        const ObjInfo& oi = op->obj[o];
        auto mat = std::make_shared<NestedMat>();
        mat->n = oi.ne + oi.nq;
        mat->ne = oi.ne;
        mat->nq = oi.nq;
        const int64_t n = mat->n;
        mat->M.alloc(size_t(n) * n);
        mat->R.alloc(size_t(n) * oi.ne);
        SLDM_CUDA(cudaMemcpyAsync(mat->M.p, Ml.p + ml_off[o], size_t(n) * n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        SLDM_CUDA(cudaMemcpyAsync(mat->R.p, Rl.p + rl_off[o], size_t(n) * oi.ne * sizeof(double2), cudaMemcpyDeviceToDevice,
                                  s));
        if (nested_setup(*mat, s)) {
          nmat[o] = mat;
        } else {
          fallback.push_back({Ml.p + ml_off[o], Rl.p + rl_off[o], int32_t(n), oi.ne});
        }
      }
      lu_solve_batched<C>(fallback, s);
    }
    for (int o = 0; o < op->nobj; ++o) {
      const int r = ref[o];
      if (!nmat[r]) continue;
      op->obj[o].nested = true;
      auto u = std::make_unique<NestedUse>();
      u->obj = o;
      u->mat_owner = r;
      u->mat = nmat[r];
      u->e0 = op->obj[o].e0;
      u->q0 = op->obj[o].q0;
      op->nested.push_back(std::move(u));
    }
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] != o || op->obj[o].nested) continue;
      const ObjInfo& oi = op->obj[o];
      // undo the length scaling of M_l: Y11 = Yh11 / l, Y21 = l Yh21
      copy_scaled<C>(Rl.p + rl_off[o], int64_t(oi.ne) * oi.ne, 1.0 / h.ell, loc + oi.oY11 * es, s);
      copy_scaled<C>(Rl.p + rl_off[o] + int64_t(oi.ne) * oi.ne, int64_t(oi.nq) * oi.ne, h.ell, loc + oi.oY21 * es, s);
    }
    // repeated objects: the first one's L^A, L^phi, K, Y11, Y21 (same layout, same sizes)
    for (int o = 0; o < op->nobj; ++o) {
      if (ref[o] == o) continue;
      const ObjInfo& oi = op->obj[o];
      const ObjInfo& ri = op->obj[ref[o]];
      const int64_t n_ee = int64_t(oi.ne) * oi.ne;
      SLDM_CUDA(cudaMemcpyAsync(loc + oi.oLA * es, loc + ri.oLA * es, n_ee * es, cudaMemcpyDeviceToDevice, s));
      SLDM_CUDA(cudaMemcpyAsync(loc + oi.oLP * es, loc + ri.oLP * es, int64_t(oi.nt) * oi.nt * es,
                                cudaMemcpyDeviceToDevice, s));
      SLDM_CUDA(cudaMemcpyAsync(loc + oi.oK * es, loc + ri.oK * es, n_ee * es, cudaMemcpyDeviceToDevice, s));
      if (oi.nested) continue;  // Y is not formed
      SLDM_CUDA(cudaMemcpyAsync(loc + oi.oY11 * es, loc + ri.oY11 * es, n_ee * es, cudaMemcpyDeviceToDevice, s));
      SLDM_CUDA(cudaMemcpyAsync(loc + oi.oY21 * es, loc + ri.oY21 * es, int64_t(oi.nq) * oi.ne * es,
                                cudaMemcpyDeviceToDevice, s));
    }
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  // ---- layered background: add the reflected part (images + tabulated remainder)
  //      to the filled blocks of L^A_m, L^phi_m, then copy the repeated ones
  if (op->layered) {
    layered_tables(op, s);
    mgf_fill_reflected<C>(m, op->H, omega, op->T, rtasks, op->LAm.p, op->ne, op->LPm.p, op->nt, s);
    copy_blocks(gr.copyA, es, op->LAm.p, op->ne, s);
    copy_blocks(gr.copyP, es, op->LPm.p, op->nt, s);
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  if (!finish) return;
  build_plans<C>(op, s);
  // ---- preconditioner P (Eq. pcext): diagonals and the per-object Schur complement inverses
  {
    std::vector<PrecObj> po;
    for (auto& oi : op->obj) po.push_back({oi.e0, oi.ne, oi.t0, oi.nt, oi.q0, 0, oi.oLA, oi.oK, oi.oLP});
    prec_setup<C>(op->pc, m, po, op->k0, op->LAm.p, op->LPm.p, op->loc.p, op->ix_val.p, s);
    op->pc.ready = true;
  }
  SLDM_CUDA(cudaStreamSynchronize(s));
}

// SLDM_PREC_F32X2: the operator filled and factored in FP64 is kept as complex64
// pairs, hi = fl32(v) and lo = fl32(v - hi), so that v = hi + lo to ~2^-48.  The
// GMRES cycles apply hi (complex64, FP32 arithmetic); the residual of iterative
// refinement applies hi + lo with compensated FP32 sums, i.e. the FP64 operator.
static void split_to_x2(sldm_op* op, cudaStream_t s) {
  auto split = [&](DBuf<char>& full, DBuf<char>& lo) {
    const int64_t n = int64_t(full.bytes() / sizeof(double2));
    DBuf<char> hi;
    hi.alloc(size_t(n) * sizeof(float2));
    lo.alloc(size_t(n) * sizeof(float2));
    split_c128(reinterpret_cast<const double2*>(full.p), n, reinterpret_cast<float2*>(hi.p),
               reinterpret_cast<float2*>(lo.p), s);
    SLDM_CUDA(cudaStreamSynchronize(s));
    std::swap(full.p, hi.p);  // full now holds hi; the complex128 copy leaves with `hi`
    std::swap(full.n, hi.n);
  };
  split(op->LAm, op->LAm_lo);
  split(op->LPm, op->LPm_lo);
  split(op->loc, op->loc_lo);
  op->prec = SLDM_PREC_F32;
  op->esz = sizeof(float2);
  op->x2 = true;
  build_plans<float2>(op, s);
  std::vector<PrecObj> po;
  for (auto& oi : op->obj) po.push_back({oi.e0, oi.ne, oi.t0, oi.nt, oi.q0, 0, oi.oLA, oi.oK, oi.oLP});
  prec_setup<float2>(op->pc, op->mesh, po, op->k0, op->LAm.p, op->LPm.p, op->loc.p, op->ix_val.p, s);
  op->pc.ready = true;
  SLDM_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- GMRES
// GMRES workspace for nr right-hand sides in lockstep (Krylov bases N x (m+1) each)
static void ensure_ws(sldm_op* op, int m, int nr) {
  if (op->ws_m == m && op->ws_nr >= nr && op->V.p) return;
  const size_t N = size_t(op->N), W = size_t(sldm_op::WR);
  op->ldv = (op->N + 63) / 64 * 64;
  op->V.alloc(size_t(op->ldv) * (m + 1) * nr);
  op->V.zero();  // the padding rows stay zero
  op->wb.alloc(N * W);
  op->wx.alloc(N * W);
  op->wr.alloc(N * W);
  op->wtmp.alloc(N * W);
  op->wtmp2.alloc(N * W);
  op->wacc.alloc(N * W);
  op->wz.alloc(N * W);
  op->dh.alloc(W * 2 * (m + 2));
  op->dnorm.alloc(W);
  // Hessenberg matrices, rotations and residual vectors on the device
  op->gH.alloc(W * size_t(m + 1) * m);
  op->gcs.alloc(W * size_t(m));
  op->gsn.alloc(W * size_t(m));
  op->gg.alloc(W * size_t(m + 1));
  op->gst.alloc(W);
  op->gscale.alloc(W);
  op->gon.alloc(W);
  op->polls.init(int(W));
  op->ws_m = m;
  op->ws_nr = nr;
}

static double dnorm(sldm_op* op, const double2* v, cudaStream_t s) {
  vnorm2(v, op->N, op->dnorm.p, s);
  double h = 0;
  SLDM_CUDA(cudaMemcpyAsync(&h, op->dnorm.p, sizeof(double), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  return std::sqrt(h);
}

// The Krylov iteration runs on the length-scaled system Dr Z Dc, Dr = diag(1,
// 1, l), Dc = diag(1/l, 1, l) (blocks j, e, u; l = mean edge length).  The
// blocks of Z scale as l (L^A), 1 (K, I_x, D), 1/l (L^phi) and 1/l^2 (k0^2), so
// the scaled system has O(1) blocks whatever the size of the geometry in
// metres, which is what the frequency scalings of the final system presume.
// With the preconditioner P of Eq. pcext applied on the right, the scaled
// preconditioner Dr P Dc cancels Dc:  operator = Dr Z P^-1 Dr^-1.
//
// Restarted, right-preconditioned GMRES for nr <= WR right-hand sides in
// lockstep: each has its own Krylov basis, Hessenberg matrix and rotations, and
// the products of one step are made together (one multi-RHS pass over the
// blocks).  Right-hand sides in op->wb, initial guesses in op->wx (N x nr);
// relres[r] = ||Dr (b_r - Z x_r)|| / ||Dr b_r||.  With `refine` (complex64
// operators) the true residual at every restart is accumulated to ~48 bits and each
// cycle stops once it has reduced that residual by REFINE_CYCLE: the cycles are
// the correction solves of iterative refinement, in the operator's precision.
// CB is the storage of the Krylov bases (complex64 for complex64 operators,
// orthogonalised in FP32); x_zero says the initial guesses are zero (the first
// residual is then b, with no product).
constexpr double REFINE_CYCLE = 1e-5;
template <class CB>
static void gmres_block(sldm_op* op, bool use_p, bool refine, bool x_zero, int m, double tol, int maxit, int nr,
                        int& iters, double* relres, cudaStream_t s) {
  const int64_t N = op->N, ne = op->ne;
  const double l = op->mesh->h.ell;
  auto col = [&](DBuf<double2>& b, int r) { return b.p + int64_t(r) * N; };
  const int64_t ldv = op->ldv;
  auto Vr = [&](int r) { return reinterpret_cast<CB*>(op->V.p) + int64_t(r) * ldv * (m + 1); };
  auto dhr = [&](int r) { return op->dh.p + int64_t(r) * 2 * (m + 2); };
  std::vector<double> bnorm(nr), beta(nr);
  for (int r = 0; r < nr; ++r) {
    vscale3(N, ne, 1.0, 1.0, l, col(op->wb, r), col(op->wb, r), s);  // bh = Dr b
    bnorm[r] = dnorm(op, col(op->wb, r), s);
    if (bnorm[r] == 0) SLDM_CUDA(cudaMemsetAsync(col(op->wx, r), 0, N * sizeof(double2), s));  // b = 0: x = 0
  }
  auto residuals = [&]() {  // wr = Dr (b - Z x), every column
    tc_check(op->tc1, s);     // a tensor-core pass whose bounded wait ran out: SLDM_ETIMEOUT
    tc_check(op->tc2, s);
    tc_check(op->pc.tc, s);
    if (x_zero) SLDM_CUDA(cudaMemsetAsync(op->wr.p, 0, size_t(nr) * N * sizeof(double2), s));  // Z 0 = 0
    else apply_any(op, op->wx.p, op->wr.p, nr, s, refine);
    x_zero = false;
    for (int r = 0; r < nr; ++r) {
      vscale3(N, ne, 1.0, 1.0, l, col(op->wr, r), col(op->wr, r), s);
      vaxpby(N, 1.0, col(op->wb, r), -1.0, col(op->wr, r), s);
      beta[r] = dnorm(op, col(op->wr, r), s);
    }
  };
  residuals();
  // Hessenberg matrices, rotations and convergence tests live on the device
  // (gmres_givens): the host learns which right-hand sides still iterate from
  // a copy of their flags that it reads without waiting, or after at most
  // LAG newer steps have been queued, so converged ones run at most LAG extra
  // (frozen) steps and the host never waits on a step it has just queued.
  constexpr int LAG = PollRing::SLOTS - 1;
  std::vector<int> it(nr, 0), kused(nr, 0);
  std::vector<char> live(nr, 0);
  std::vector<GmresState> hst(nr);
  PollRing& polls = op->polls;
  for (;;) {
    std::vector<int> act;
    for (int r = 0; r < nr; ++r) {
      SLDM_REQUIRE(std::isfinite(beta[r]), SLDM_ENUMERIC, "GMRES: non-finite residual");
      if (bnorm[r] > 0 && beta[r] / bnorm[r] > tol && it[r] < maxit) act.push_back(r);
    }
    if (act.empty()) break;
    {
      std::vector<double2> g0(size_t(nr) * (m + 1), make_double2(0.0, 0.0));
      for (int r = 0; r < nr; ++r) {
        hst[r] = GmresState{it[r], 0, 0, 0, bnorm[r], beta[r]};
        g0[size_t(r) * (m + 1)] = make_double2(beta[r], 0.0);
      }
      for (int r : act) {
        vaxpby<double2, CB>(N, 1.0 / beta[r], col(op->wr, r), 0.0, Vr(r), s);
        hst[r].live = 1;
        live[r] = 1;
        kused[r] = 0;
      }
      SLDM_CUDA(cudaMemcpyAsync(op->gg.p, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, s));
      SLDM_CUDA(cudaMemcpyAsync(op->gst.p, hst.data(), nr * sizeof(GmresState), cudaMemcpyHostToDevice, s));
      SLDM_CUDA(cudaStreamSynchronize(s));  // g0, hst are host temporaries
    }
    std::vector<int> on, on_dev;
    int next_poll = 0, oldest = 0;  // ring of outstanding flag copies [oldest, next_poll)
    auto consume = [&](bool wait) {
      while (oldest < next_poll) {
        const int sl = oldest % PollRing::SLOTS;
        if (!wait) {
          const cudaError_t q = cudaEventQuery(polls.ev[sl]);
          if (q == cudaErrorNotReady) break;
          SLDM_CUDA(q);
        } else {
          SLDM_CUDA(cudaEventSynchronize(polls.ev[sl]));
        }
        for (int r : act)
          if (!polls.flags[sl][r]) live[r] = 0;
        ++oldest;
        wait = false;  // one forced wait at most
      }
    };
    for (int k = 0; k < m; ++k) {
      on.clear();
      for (int r : act)
        if (live[r]) on.push_back(r);
      if (on.empty()) break;
      const int na = int(on.size());
      if (on != on_dev) {
        SLDM_CUDA(cudaMemcpyAsync(op->gon.p, on.data(), na * sizeof(int), cudaMemcpyHostToDevice, s));
        SLDM_CUDA(cudaStreamSynchronize(s));  // `on` is reused by the host
        on_dev = on;
      }
      // the products of this step, together: w_r = Dr Z P^-1 Dr^-1 v_r (or Dr Z Dc v_r)
      VecBatch<CB, double2> bv;
      for (int j = 0; j < na; ++j) {
        bv.x[j] = Vr(on[j]) + int64_t(k) * ldv;
        bv.y[j] = col(use_p ? op->wtmp2 : op->wtmp, j);
        bv.a[j] = 1.0;
      }
      if (use_p) {
        vscale3_batch(N, ne, 1.0, 1.0, 1.0 / l, bv, na, s);
        prec_apply(op->pc, op->mesh, op->wtmp2.p, op->wtmp.p, N, na, s);
      } else {
        vscale3_batch(N, ne, 1.0 / l, 1.0, l, bv, na, s);
      }
      apply_any(op, op->wtmp.p, op->wz.p, na, s);
      {
        // classical Gram-Schmidt, twice, of every w_r = Dr wz_r against its basis
        ScopedTimer tgs("gram_schmidt", s);
        SLDM_CUDA(cudaMemsetAsync(op->dh.p, 0, op->dh.bytes(), s));
        SLDM_CUDA(cudaMemsetAsync(op->dnorm.p, 0, op->dnorm.bytes(), s));
        VecBatch<double2, CB> bw;
        KrylovStep ks;
        ks.n = N;
        ks.ldv = ldv;
        ks.k = k + 1;
        ks.na = na;
        ks.nrm = op->dnorm.p;
        for (int j = 0; j < na; ++j) {
          bw.x[j] = col(op->wz, j);
          bw.y[j] = Vr(on[j]) + int64_t(k + 1) * ldv;
          bw.a[j] = 1.0;
          ks.V[j] = Vr(on[j]);
          ks.h[j] = dhr(on[j]);
        }
        vscale3_batch(N, ne, 1.0, 1.0, l, bw, na, s);
        // bytes the two passes move: per pass V[:, :k+1] read by the dots and by the
        // update, w read by both and written by the update
        timer_units("gram_schmidt", double(na) * 2.0 * (2.0 * (k + 1) + 3.0) * double(ldv) * sizeof(CB));
        krylov_dots<CB>(ks, s);
        krylov_update<CB>(ks, false, s);
        for (int j = 0; j < na; ++j) ks.h[j] = dhr(on[j]) + (m + 2);
        krylov_dots<CB>(ks, s);
        krylov_update<CB>(ks, true, s);
      }
      // rotations and convergence tests on the device; v_{k+1} = w / h_{k+1,k}
      GivensArgs ga{};
      ga.k = k;
      ga.m = m;
      ga.na = na;
      ga.refine = refine ? 1 : 0;
      ga.on = op->gon.p;
      ga.dh = op->dh.p;
      ga.ldh = 2 * (m + 2);
      ga.nrm = op->dnorm.p;
      ga.H = op->gH.p;
      ga.cs = op->gcs.p;
      ga.sn = op->gsn.p;
      ga.g = op->gg.p;
      ga.st = op->gst.p;
      ga.tol = tol;
      ga.cycle = REFINE_CYCLE;
      ga.maxit = maxit;
      ga.scale = op->gscale.p;
      gmres_givens(ga, s);
      VecBatch<CB, CB> bn;
      for (int j = 0; j < na; ++j) bn.x[j] = bn.y[j] = Vr(on[j]) + int64_t(k + 1) * ldv;
      vscale_dev_batch<CB>(N, bn, op->gscale.p, na, s);
      // queue a copy of the flags; read the finished copies, waiting only when LAG are pending
      {
        if (next_poll - oldest == PollRing::SLOTS) consume(true);
        const int sl = next_poll % PollRing::SLOTS;
        SLDM_CUDA(cudaMemcpy2DAsync(polls.flags[sl], sizeof(int32_t), &op->gst.p[0].live, sizeof(GmresState),
                                    sizeof(int32_t), nr, cudaMemcpyDeviceToHost, s));
        SLDM_CUDA(cudaEventRecord(polls.ev[sl], s));
        ++next_poll;
        consume(next_poll - oldest > LAG);
      }
    }
    // the cycle's state; y = H^-1 g on the device;  x += (P^-1 Dr^-1 or Dc) V y
    SLDM_CUDA(cudaMemcpyAsync(hst.data(), op->gst.p, nr * sizeof(GmresState), cudaMemcpyDeviceToHost, s));
    SLDM_CUDA(cudaStreamSynchronize(s));
    for (int r : act) {
      it[r] = hst[r].it;
      kused[r] = hst[r].kused;
    }
    std::vector<int> solve;
    for (int r : act)
      if (kused[r] > 0) solve.push_back(r);
    if (!solve.empty()) {
      SLDM_CUDA(cudaMemcpyAsync(op->gon.p, solve.data(), solve.size() * sizeof(int), cudaMemcpyHostToDevice, s));
      gmres_backsolve(int(solve.size()), op->gon.p, m, op->gH.p, op->gg.p, op->gst.p, op->dh.p, 2 * (m + 2), s);
      SLDM_CUDA(cudaStreamSynchronize(s));  // `solve` is a host temporary
    }
    for (int r : solve) {
      const int ku = kused[r];
      SLDM_CUDA(cudaMemsetAsync(col(op->wacc, r), 0, N * sizeof(double2), s));
      vmul<CB, double2>(Vr(r), ldv, ku, dhr(r), 1.0, col(op->wacc, r), N, s);
      if (use_p) {
        vscale3(N, ne, 1.0, 1.0, 1.0 / l, col(op->wacc, r), col(op->wtmp2, 0), s);
        prec_apply(op->pc, op->mesh, col(op->wtmp2, 0), col(op->wtmp, 0), N, 1, s);
      } else {
        vscale3(N, ne, 1.0 / l, 1.0, l, col(op->wacc, r), col(op->wtmp, 0), s);
      }
      vaxpby(N, 1.0, col(op->wtmp, 0), 1.0, col(op->wx, r), s);
    }
    residuals();
  }
  for (int r = 0; r < nr; ++r) {
    relres[r] = bnorm[r] > 0 ? beta[r] / bnorm[r] : 0.0;
    iters += it[r];
  }
}

}  // namespace sldm

using namespace sldm;

#define API_BEGIN try {
#define API_END                            \
  }                                        \
  catch (const sldm::Error& e) {           \
    sldm::set_error(e.msg);                \
    return e.code;                         \
  }                                        \
  catch (const std::exception& e) {        \
    sldm::set_error(e.what());             \
    return SLDM_EINVAL;                    \
  }                                        \
  return SLDM_OK;

extern "C" {

void sldm_last_error(char* buf, size_t len) {
  if (!buf || len == 0) return;
  std::strncpy(buf, g_err.c_str(), len - 1);
  buf[len - 1] = 0;
}

int sldm_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* obj_id,
                     sldm_mesh** out) {
  API_BEGIN
  SLDM_REQUIRE(out, SLDM_EINVAL, "mesh_create: out is null");
  *out = nullptr;
  auto* m = new sldm_mesh();
  try {
    build_host_mesh(xyz, nv, tri, nt, obj_id, m->h);
    SLDM_CUDA(cudaGetDevice(&m->device));
    const HostMesh& h = m->h;
    DevMesh& d = m->d;
    d.xyz.upload(h.xyz);
    d.tri.upload(h.tri);
    d.tri_edge.upload(h.tri_edge);
    d.tri_sign.upload(h.tri_sign);
    d.tplus.upload(h.tplus);
    d.tminus.upload(h.tminus);
    d.obj.upload(h.obj);
    std::vector<int32_t> q2t;
    for (int64_t t = 0; t < h.nt; ++t)
      if (t + 1 != h.tri_begin[h.obj[t] + 1]) q2t.push_back(int32_t(t));
    d.q2t.upload(q2t);
    d.tri_begin.upload(h.tri_begin);
    d.edge_begin.upload(h.edge_begin);
    d.btri_edge.upload(h.btri_edge);
    d.btri_sign.upload(h.btri_sign);
    d.bc_ptr.upload(h.bc_ptr);
    d.bc_row.upload(h.bc_row);
    d.bc_val.upload(h.bc_val);
    d.touchL_a.upload(h.touchL_a);
    d.touchL_b.upload(h.touchL_b);
    d.touchK_a.upload(h.touchK_a);
    d.touchK_c.upload(h.touchK_c);
    d.ix_ptr.upload(h.ix_ptr);
    d.ix_col.upload(h.ix_col);
    d.ixc_ptr.upload(h.ixc_ptr);
    d.ixc_tri.upload(h.ixc_tri);
    d.ixc_child.upload(h.ixc_child);
    d.ixc_i.upload(h.ixc_i);
    d.ixc_j.upload(h.ixc_j);
    d.ixc_coef.upload(h.ixc_coef);
    geometry(h, d, 0);
    SLDM_CUDA(cudaStreamSynchronize(0));
  } catch (...) {
    delete m;
    throw;
  }
  *out = m;
  API_END
}

int sldm_mesh_info_get(const sldm_mesh* m, sldm_mesh_info* info) {
  API_BEGIN
  SLDM_REQUIRE(m && info, SLDM_EINVAL, "mesh_info: null argument");
  info->nv = m->h.nv;
  info->nt = m->h.nt;
  info->ne = m->h.ne;
  info->nobj = m->h.nobj;
  info->n_unknowns = 2 * m->h.ne + m->h.nt - m->h.nobj;
  info->n_bary_edges = m->h.nbe;
  API_END
}

int sldm_mesh_edges(const sldm_mesh* m, int64_t* uv, int64_t* tplus, int64_t* tminus) {
  API_BEGIN
  SLDM_REQUIRE(m, SLDM_EINVAL, "mesh_edges: null mesh");
  for (int64_t n = 0; n < m->h.ne; ++n) {
    if (uv) {
      uv[2 * n] = m->h.uv[2 * n];
      uv[2 * n + 1] = m->h.uv[2 * n + 1];
    }
    if (tplus) tplus[n] = m->h.tplus[n];
    if (tminus) tminus[n] = m->h.tminus[n];
  }
  API_END
}

int sldm_mesh_destroy(sldm_mesh* m) {
  API_BEGIN
  delete m;
  API_END
}

int sldm_stack_create(const sldm_layer* layers, int32_t nlayers, double z_top, int32_t bottom, sldm_stack** out) {
  API_BEGIN
  SLDM_REQUIRE(out && layers && nlayers >= 1, SLDM_EINVAL, "stack_create: invalid arguments");
  *out = nullptr;
  SLDM_REQUIRE(nlayers <= MGF_MAX_LAYERS, SLDM_ENOTSUP, "stack_create: too many layers");
  SLDM_REQUIRE(bottom == SLDM_BOTTOM_HALFSPACE || bottom == SLDM_BOTTOM_PEC, SLDM_EINVAL, "stack_create: unknown bottom");
  SLDM_REQUIRE(std::isfinite(z_top), SLDM_EINVAL, "stack_create: z_top must be finite");
  for (int i = 0; i < nlayers; ++i) {
    SLDM_REQUIRE(layers[i].eps_r > 0 && layers[i].mu_r > 0 && layers[i].sigma >= 0 && std::isfinite(layers[i].eps_r) &&
                     std::isfinite(layers[i].mu_r) && std::isfinite(layers[i].sigma),
                 SLDM_EINVAL, "stack_create: invalid layer material");
    const bool finite = i > 0 && (bottom == SLDM_BOTTOM_PEC || i < nlayers - 1);
    SLDM_REQUIRE(!finite || (layers[i].thickness > 0 && std::isfinite(layers[i].thickness)), SLDM_EINVAL,
                 "stack_create: finite layers need a positive thickness");
  }
  auto* st = new sldm_stack();
  st->layers.assign(layers, layers + nlayers);
  st->z_top = z_top;
  st->bottom = bottom;
  *out = st;
  API_END
}

int sldm_stack_destroy(sldm_stack* s) {
  API_BEGIN
  delete s;
  API_END
}

int sldm_assemble(const sldm_mesh* m, const sldm_stack* st, const sldm_material* per_obj, double freq_hz,
                  const sldm_assemble_opts* opts, sldm_op** out) {
  API_BEGIN
  SLDM_REQUIRE(m && st && per_obj && out, SLDM_EINVAL, "assemble: null argument");
  SLDM_REQUIRE(freq_hz > 0 && std::isfinite(freq_hz), SLDM_EINVAL, "assemble: frequency must be positive");
  *out = nullptr;
  int dev = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  SLDM_REQUIRE(dev == m->device, SLDM_EINVAL, "assemble: current device differs from the mesh's device");
  for (int64_t o = 0; o < m->h.nobj; ++o)
    SLDM_REQUIRE(per_obj[o].eps_r > 0 && per_obj[o].mu_r > 0 && per_obj[o].sigma >= 0 &&
                     std::isfinite(per_obj[o].eps_r) && std::isfinite(per_obj[o].mu_r) && std::isfinite(per_obj[o].sigma),
                 SLDM_EINVAL, "assemble: invalid object material");
  auto* op = new sldm_op();
  try {
    op->mesh = m;
    const int prec = opts ? opts->precision : SLDM_PREC_F64;
    SLDM_REQUIRE(prec == SLDM_PREC_F64 || prec == SLDM_PREC_F32 || prec == SLDM_PREC_F32X2, SLDM_EINVAL,
                 "assemble: unknown precision");
    op->prec = prec == SLDM_PREC_F32 ? SLDM_PREC_F32 : SLDM_PREC_F64;  // X2 fills in FP64, then splits
    op->want_x2 = prec == SLDM_PREC_F32X2;
    if (opts && opts->nested_min != 0) op->nested_min = opts->nested_min;
    op->esz = op->prec == SLDM_PREC_F32 ? 8 : 16;
    op->freq = freq_hz;
    op->device = dev;
    op->k0 = 2 * PI_ * freq_hz / C0_;
    op->ne = m->h.ne;
    op->nt = m->h.nt;
    op->nobj = m->h.nobj;
    op->nq = op->nt - op->nobj;
    op->N = 2 * op->ne + op->nq;
    const int nl = int(st->layers.size());
    op->layered = nl > 1 || st->bottom == SLDM_BOTTOM_PEC;
    int lay = 0;
    if (op->layered) {
      lay = per_obj[0].layer;
      for (int64_t o = 0; o < m->h.nobj; ++o)
        SLDM_REQUIRE(per_obj[o].layer == lay, SLDM_ENOTSUP, "assemble: every object must lie in the same layer");
      SLDM_REQUIRE(lay >= 0 && lay < nl, SLDM_EINVAL, "assemble: layer index out of range");
      // layer bounds: layer 0 above z_top; finite layers below, top to bottom
      MgfStackHost& H = op->H;
      H.l = lay;
      H.pec = st->bottom == SLDM_BOTTOM_PEC;
      op->thick.assign(nl, 0.0);
      double z = st->z_top, zb = -1e300, zu = 1e300;
      for (int i = 0; i < nl; ++i) {
        H.eps.push_back(eps_complex(st->layers[i].eps_r, st->layers[i].sigma, 2 * PI_ * freq_hz));
        H.mu.push_back(st->layers[i].mu_r);
        const bool finite = i > 0 && (H.pec || i < nl - 1);
        op->thick[i] = finite ? st->layers[i].thickness : 0.0;
        H.d.push_back(op->thick[i]);
        const double top = i == 0 ? 1e300 : z;
        const double bot = i == 0 ? st->z_top : (finite ? z - op->thick[i] : -1e300);
        if (i == lay) {
          zb = bot;
          zu = top;
        }
        if (i > 0 && finite) z -= op->thick[i];
      }
      H.zb = zb;
      H.zu = zu;
      H.top = lay > 0;
      H.bot = zb > -1e299;
      op->z_top = st->z_top;
      // objects lie inside their layer and may rest on its interfaces (to 1e-9 of the mesh size)
      double span = 0;
      for (int d = 0; d < 3; ++d) {
        double a = 1e300, b = -1e300;
        for (int64_t v = 0; v < m->h.nv; ++v) {
          a = std::min(a, m->h.xyz[3 * v + d]);
          b = std::max(b, m->h.xyz[3 * v + d]);
        }
        span = std::max(span, b - a);
      }
      const double tol = 1e-9 * span;
      for (int64_t v = 0; v < m->h.nv; ++v)
        SLDM_REQUIRE(m->h.xyz[3 * v + 2] >= zb - tol && m->h.xyz[3 * v + 2] <= zu + tol, SLDM_EINVAL,
                     "assemble: the objects must lie inside their layer (they may rest on an interface)");
    }
    const sldm_layer& L = st->layers[lay];
    op->eps_b = eps_complex(L.eps_r, L.sigma, 2 * PI_ * freq_hz);
    op->mu_b = L.mu_r;
    op->kb = op->k0 * std::sqrt(op->eps_b * op->mu_b);
    cudaStream_t s = opts ? (cudaStream_t)opts->stream : 0;
    ScopedTimer tm("assemble", s);
    if (op->prec == SLDM_PREC_F32) {
      assemble_impl<float>(op, per_obj, s);
    } else if (prec == SLDM_PREC_F32X2) {
      assemble_impl<double>(op, per_obj, s, false);
      split_to_x2(op, s);
    } else {
      assemble_impl<double>(op, per_obj, s);
    }
  } catch (...) {
    delete op;
    throw;
  }
  *out = op;
  API_END
}

int sldm_op_info_get(const sldm_op* op, sldm_op_info* info) {
  API_BEGIN
  SLDM_REQUIRE(op && info, SLDM_EINVAL, "op_info: null argument");
  info->n_unknowns = op->N;
  info->ne = op->ne;
  info->nt = op->nt;
  info->nobj = op->nobj;
  info->device_bytes = op_bytes(op);
  info->precision = op->x2 ? SLDM_PREC_F32X2 : op->prec;
  info->tc_from = op->prec == SLDM_PREC_F32 ? op->plan2.tc_from : 0;
  info->k0 = op->k0;
  API_END
}

int sldm_op_block(const sldm_op* op, int32_t which, int32_t obj, void* dst, int32_t where, int64_t* rows, int64_t* cols) {
  API_BEGIN
  SLDM_REQUIRE(op, SLDM_EINVAL, "op_block: null op");
  const bool global = which == SLDM_BLOCK_LAM || which == SLDM_BLOCK_LPM || which == SLDM_BLOCK_IX;
  SLDM_REQUIRE(global || (obj >= 0 && obj < op->nobj), SLDM_EINVAL, "op_block: object index out of range");
  SLDM_REQUIRE(which != SLDM_BLOCK_KBAR_L, SLDM_ENOTSUP, "op_block: Kbar_l is not retained after assembly");
  int64_t r = 0, c = 0;
  const char* src = nullptr;
  const ObjInfo* oi = global ? nullptr : &op->obj[obj];
  switch (which) {
    case SLDM_BLOCK_LAM: r = c = op->ne; src = op->LAm.p; break;
    case SLDM_BLOCK_LPM: r = c = op->nt; src = op->LPm.p; break;
    case SLDM_BLOCK_IX: r = c = op->ne; break;
    case SLDM_BLOCK_LA: r = c = oi->ne; src = op->loc.p + oi->oLA * op->esz; break;
    case SLDM_BLOCK_LP: r = c = oi->nt; src = op->loc.p + oi->oLP * op->esz; break;
    case SLDM_BLOCK_K: r = c = oi->ne; src = op->loc.p + oi->oK * op->esz; break;
    case SLDM_BLOCK_Y11:
      SLDM_REQUIRE(!oi->nested, SLDM_ENOTSUP, "op_block: Y is applied by inner solves for this object (not formed)");
      r = c = oi->ne; src = op->loc.p + oi->oY11 * op->esz; break;
    case SLDM_BLOCK_Y21:
      SLDM_REQUIRE(!oi->nested, SLDM_ENOTSUP, "op_block: Y is applied by inner solves for this object (not formed)");
      r = oi->nq; c = oi->ne; src = op->loc.p + oi->oY21 * op->esz; break;
    default: SLDM_REQUIRE(false, SLDM_EINVAL, "op_block: unknown block");
  }
  if (rows) *rows = r;
  if (cols) *cols = c;
  if (!dst) return SLDM_OK;
  const int64_t n = r * c;
  std::vector<double2> host;
  if (which == SLDM_BLOCK_IX) {
    host.assign(size_t(n), make_double2(0, 0));
    std::vector<double> v(op->mesh->h.ix_col.size());
    SLDM_CUDA(cudaMemcpy(v.data(), op->ix_val.p, v.size() * sizeof(double), cudaMemcpyDeviceToHost));
    for (int64_t mrow = 0; mrow < op->ne; ++mrow)
      for (int z = op->mesh->h.ix_ptr[mrow]; z < op->mesh->h.ix_ptr[mrow + 1]; ++z)
        host[size_t(mrow * op->ne + op->mesh->h.ix_col[z])].x = v[z];
    if (where == SLDM_HOST) std::memcpy(dst, host.data(), n * sizeof(double2));
    else SLDM_CUDA(cudaMemcpy(dst, host.data(), n * sizeof(double2), cudaMemcpyHostToDevice));
    return SLDM_OK;
  }
  DBuf<double2> tmp;
  double2* d = (where == SLDM_DEVICE) ? (double2*)dst : nullptr;
  if (!d) {
    tmp.alloc(n);
    d = tmp.p;
  }
  if (op->prec == SLDM_PREC_F32) {
    to_c128<float2>(src, n, d, 0);
    if (op->x2) {  // the FP64 value: hi + lo
      const char* lo = which == SLDM_BLOCK_LAM   ? op->LAm_lo.p
                       : which == SLDM_BLOCK_LPM ? op->LPm_lo.p
                                                 : op->loc_lo.p + (src - op->loc.p);
      add_lo_c128(reinterpret_cast<const float2*>(lo), n, d, 0);
    }
  } else {
    to_c128<double2>(src, n, d, 0);
  }
  if (where == SLDM_HOST) SLDM_CUDA(cudaMemcpy(dst, d, n * sizeof(double2), cudaMemcpyDeviceToHost));
  SLDM_CUDA(cudaDeviceSynchronize());
  API_END
}

int sldm_op_table(const sldm_op* op, int32_t which, void* dst, int64_t* dims, double* grid) {
  API_BEGIN
  SLDM_REQUIRE(op, SLDM_EINVAL, "op_table: null op");
  SLDM_REQUIRE(op->layered, SLDM_EINVAL, "op_table: the operator has a homogeneous background");
  SLDM_REQUIRE(which == 0 || which == 1, SLDM_EINVAL, "op_table: which must be 0 (z + z') or 1 (z - z')");
  const int n2 = which == 0 ? op->T.ns : op->T.nd;
  if (dims) {
    dims[0] = 5;
    dims[1] = op->T.nr;
    dims[2] = n2;
  }
  if (grid) {
    grid[0] = op->T.lr0;
    grid[1] = op->T.lr1;
    grid[2] = op->T.s0;
    grid[3] = op->T.s1;
    grid[4] = op->T.d1;
  }
  if (dst)
    SLDM_CUDA(cudaMemcpy(dst, which == 0 ? op->T.A.p : op->T.B.p, size_t(5) * op->T.nr * n2 * sizeof(double2),
                         cudaMemcpyDeviceToHost));
  API_END
}

int sldm_op_destroy(sldm_op* op) {
  API_BEGIN
  delete op;
  API_END
}

int sldm_apply(const sldm_op* op, const void* x, void* y, int32_t nrhs, int32_t where, void* stream) {
  API_BEGIN
  SLDM_REQUIRE(op && x && y && nrhs >= 1, SLDM_EINVAL, "apply: invalid arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t bytes = size_t(op->N) * nrhs * sizeof(double2);
  // SLDM_PREC_F32X2: the product of the FP64 operator (hi + lo, compensated FP32 sums)
  if (where == SLDM_DEVICE) {
    apply_any(op, (const double2*)x, (double2*)y, nrhs, s, op->x2);
  } else {
    DBuf<double2> dx, dy;
    dx.alloc(size_t(op->N) * nrhs);
    dy.alloc(size_t(op->N) * nrhs);
    SLDM_CUDA(cudaMemcpyAsync(dx.p, x, bytes, cudaMemcpyHostToDevice, s));
    apply_any(op, dx.p, dy.p, nrhs, s, op->x2);
    SLDM_CUDA(cudaMemcpyAsync(y, dy.p, bytes, cudaMemcpyDeviceToHost, s));
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  API_END
}

int sldm_rhs_planewave(const sldm_op* op, const double* khat, const double* pol, int32_t nrhs, void* b, int32_t where,
                       void* stream) {
  API_BEGIN
  SLDM_REQUIRE(op && khat && pol && b && nrhs >= 1, SLDM_EINVAL, "rhs_planewave: invalid arguments");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<double> kp(size_t(6) * nrhs);
  for (int r = 0; r < nrhs; ++r)
    for (int d = 0; d < 3; ++d) {
      kp[6 * r + d] = khat[3 * r + d];
      kp[6 * r + 3 + d] = pol[3 * r + d];
    }
  DBuf<double> dk;
  dk.upload(kp, s);
  DBuf<double2> tmp;
  double2* db = (where == SLDM_DEVICE) ? (double2*)b : nullptr;
  if (!db) {
    tmp.alloc(size_t(op->N) * nrhs);
    db = tmp.p;
  }
  SLDM_CUDA(cudaMemsetAsync(db, 0, size_t(op->N) * nrhs * sizeof(double2), s));
  if (op->layered) {
    for (int r = 0; r < nrhs; ++r)
      SLDM_REQUIRE(khat[3 * r + 2] < 0, SLDM_EINVAL, "rhs_planewave: layered backgrounds take incidence from the top (khat_z < 0)");
    std::vector<double> rec(size_t(PW_REC) * nrhs);
    for (int r = 0; r < nrhs; ++r)
      mgf_plane_wave(op->H, op->thick, op->z_top, 2 * PI_ * op->freq, khat + 3 * r, pol + 3 * r, rec.data() + size_t(PW_REC) * r);
    DBuf<double> drec;
    drec.upload(rec, s);
    rhs_planewave_layered(op->mesh, drec.p, nrhs, db, op->N, s);
  } else {
    rhs_planewave(op->mesh, op->k0, dk.p, nrhs, db, op->N, s);
  }
  if (where == SLDM_HOST)
    SLDM_CUDA(cudaMemcpyAsync(b, db, size_t(op->N) * nrhs * sizeof(double2), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  API_END
}

int sldm_solve(const sldm_op* op_, const void* b, void* x, int32_t nrhs, const sldm_solve_opts* opts,
               sldm_solve_info* info, int32_t where, void* stream) {
  API_BEGIN
  SLDM_REQUIRE(op_ && b && x && nrhs >= 1, SLDM_EINVAL, "solve: invalid arguments");
  sldm_op* op = const_cast<sldm_op*>(op_);
  std::unique_lock<std::mutex> lock(op->busy, std::try_to_lock);
  SLDM_REQUIRE(lock.owns_lock(), SLDM_EBUSY, "solve: operator in use by another thread");
  double tol = (opts && opts->tol > 0) ? opts->tol : 1e-8;
  int m = (opts && opts->restart > 0) ? opts->restart : 300;
  m = int(std::min<int64_t>(m, op->N));
  SLDM_REQUIRE(m <= 1000, SLDM_EINVAL, "solve: restart length above 1000");
  int maxit = (opts && opts->maxit > 0) ? opts->maxit : 2000;
  bool x0 = opts && opts->x0_given;
  bool use_p = !(opts && opts->precond == SLDM_PRECOND_NONE) && op->pc.ready;
  bool refine = op->prec == SLDM_PREC_F32 && !(opts && opts->refine == SLDM_REFINE_OFF);
  cudaStream_t s = (cudaStream_t)stream;
  const int W = sldm_op::WR;
  ensure_ws(op, m, std::min<int>(nrhs, W));
  const size_t vb = size_t(op->N) * sizeof(double2);
  int iters = 0;
  double worst = 0;
  for (int r0 = 0; r0 < nrhs; r0 += W) {
    const int nr = std::min(W, nrhs - r0);
    const char* br = (const char*)b + r0 * vb;
    char* xr = (char*)x + r0 * vb;
    cudaMemcpyKind k_in = where == SLDM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    SLDM_CUDA(cudaMemcpyAsync(op->wb.p, br, nr * vb, k_in, s));
    if (x0) SLDM_CUDA(cudaMemcpyAsync(op->wx.p, xr, nr * vb, k_in, s));
    else SLDM_CUDA(cudaMemsetAsync(op->wx.p, 0, nr * vb, s));
    double rel[sldm_op::WR];
    {
      ScopedTimer tm("gmres", s);
      // complex64 operators keep the Krylov basis in complex64 and orthogonalise
      // in FP32 (the cycles are correction solves; the residual that decides
      // convergence is formed in FP64 at each restart when refining)
      if (op->prec == SLDM_PREC_F32) gmres_block<float2>(op, use_p, refine, !x0, m, tol, maxit, nr, iters, rel, s);
      else gmres_block<double2>(op, use_p, refine, !x0, m, tol, maxit, nr, iters, rel, s);
    }
    for (int r = 0; r < nr; ++r) worst = std::max(worst, rel[r]);
    cudaMemcpyKind k_out = where == SLDM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    SLDM_CUDA(cudaMemcpyAsync(xr, op->wx.p, nr * vb, k_out, s));
  }
  SLDM_CUDA(cudaStreamSynchronize(s));
  if (info) {
    info->iters = iters;
    info->relres = worst;
    info->status = worst <= tol ? SLDM_OK : SLDM_ENOTCONV;
  }
  if (worst > tol) {
    set_error("solve: GMRES did not reach the tolerance");
    return SLDM_ENOTCONV;
  }
  API_END
}

int sldm_port_rhs(const sldm_op* op, int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs,
                  const double* V, int32_t ncols, void* b, int32_t where, void* stream) {
  API_BEGIN
  SLDM_REQUIRE(op && V && b && ncols >= 1, SLDM_EINVAL, "port_rhs: invalid arguments");
  port_check(op->mesh->h, nports, ring_ptr, edges, signs);
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<double2> tmp;
  double2* db = (where == SLDM_DEVICE) ? (double2*)b : nullptr;
  if (!db) {
    tmp.alloc(size_t(op->N) * ncols);
    db = tmp.p;
  }
  SLDM_CUDA(cudaMemsetAsync(db, 0, size_t(op->N) * ncols * sizeof(double2), s));
  port_rhs(nports, ring_ptr, edges, signs, reinterpret_cast<const double2*>(V), ncols, db, op->N, s);
  if (where == SLDM_HOST)
    SLDM_CUDA(cudaMemcpyAsync(b, db, size_t(op->N) * ncols * sizeof(double2), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  API_END
}

int sldm_port_currents(const sldm_op* op, int32_t nports, const int32_t* ring_ptr, const int32_t* edges,
                       const int8_t* signs, const void* x, int32_t ncols, double* I, int32_t where, void* stream) {
  API_BEGIN
  SLDM_REQUIRE(op && x && I && ncols >= 1, SLDM_EINVAL, "port_currents: invalid arguments");
  port_check(op->mesh->h, nports, ring_ptr, edges, signs);
  cudaStream_t s = (cudaStream_t)stream;
  DBuf<double2> tmp;
  const double2* dx = (where == SLDM_DEVICE) ? (const double2*)x : nullptr;
  if (!dx) {
    tmp.alloc(size_t(op->N) * ncols);
    SLDM_CUDA(cudaMemcpyAsync(tmp.p, x, size_t(op->N) * ncols * sizeof(double2), cudaMemcpyHostToDevice, s));
    dx = tmp.p;
  }
  port_currents(nports, ring_ptr, edges, signs, dx, op->N, ncols, op->k0, reinterpret_cast<double2*>(I), s);
  API_END
}

int sldm_farfield_n(const sldm_op* op_, const void* x, int32_t nrhs, int32_t where, const double* theta, const double* phi,
                    int32_t n, double* rcs) {
  API_BEGIN
  SLDM_REQUIRE(op_ && x && theta && phi && rcs && n >= 1 && nrhs >= 1, SLDM_EINVAL, "farfield: invalid arguments");
  sldm_op* op = const_cast<sldm_op*>(op_);
  if (op->layered)
    for (int i = 0; i < n; ++i)
      SLDM_REQUIRE(theta[i] >= 0 && theta[i] < 0.5 * PI_, SLDM_EINVAL,
                   "farfield: above a stack, observation directions in the upper half-space only (theta < pi/2)");
  cudaStream_t s = 0;
  ScopedTimer tm("farfield", s);
  const int WR = sldm_op::WR;
  const int nr_pass = std::min(nrhs, WR);
  DBuf<double2> dx, jd;
  dx.alloc(size_t(op->N) * nr_pass);
  jd.alloc(size_t(op->ne) * nrhs);
  ApplyDims D{int32_t(op->ne), int32_t(op->nt), int32_t(op->nq), int32_t(op->nobj)};
  // j_Delta = j - Y11 e (per object), from the first two stages of the structured product
  for (int r0 = 0; r0 < nrhs; r0 += WR) {
    const int nr = std::min(WR, nrhs - r0);
    const size_t bytes = size_t(op->N) * nr * sizeof(double2);
    const char* xs = static_cast<const char*>(x) + size_t(op->N) * r0 * sizeof(double2);
    SLDM_CUDA(cudaMemcpyAsync(dx.p, xs, bytes, where == SLDM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    if (op->prec == SLDM_PREC_F32) {
      apply_glue_split<float2>(dx.p, op->N, D, op->wj.p, op->we.p, op->wu.p, nr, s);
      gemv_jobs<float2>(op->plan1, nr, s);
      apply_glue_prep<float2>(op->mesh, D, op->wj.p, op->wu.p, op->wt1.p, op->wt2.p, op->wa.p, op->wc.p, op->wbc.p,
                              op->wbu.p, nr, s, op->mesh->d.tri_begin.p, op->mesh->d.edge_begin.p);
      to_c128<float2>(op->wa.p, int64_t(op->ne) * nr, jd.p + int64_t(op->ne) * r0, s);
    } else {
      apply_glue_split<double2>(dx.p, op->N, D, op->wj.p, op->we.p, op->wu.p, nr, s);
      gemv_jobs<double2>(op->plan1, nr, s);
      for (const auto& u : op->nested)  // objects whose Y E comes from inner solves
        nested_apply(*u, op->wnt.p, op->wny.p, op->wnr.p, op->ldn, reinterpret_cast<double2*>(op->wt1.p), op->ne,
                     reinterpret_cast<double2*>(op->wt2.p), op->nq, nr, op->mesh->h.ell, s);
      apply_glue_prep<double2>(op->mesh, D, op->wj.p, op->wu.p, op->wt1.p, op->wt2.p, op->wa.p, op->wc.p, op->wbc.p,
                               op->wbu.p, nr, s, op->mesh->d.tri_begin.p, op->mesh->d.edge_begin.p);
      to_c128<double2>(op->wa.p, int64_t(op->ne) * nr, jd.p + int64_t(op->ne) * r0, s);
    }
  }
  DBuf<double> da, dr;
  dr.alloc(size_t(n) * nrhs);
  if (op->layered) {
    // reciprocity: the stack's theta- and phi-polarised waves arriving from each direction
    std::vector<double> rec(size_t(2) * n * PW_REC);
    for (int i = 0; i < n; ++i) {
      const double st = std::sin(theta[i]), ct = std::cos(theta[i]), sp = std::sin(phi[i]), cp = std::cos(phi[i]);
      const double khat[3] = {-st * cp, -st * sp, -ct};
      const double pt[3] = {ct * cp, ct * sp, -st}, pp[3] = {-sp, cp, 0.0};
      mgf_plane_wave(op->H, op->thick, op->z_top, 2 * PI_ * op->freq, khat, pt, rec.data() + size_t(2 * i) * PW_REC);
      mgf_plane_wave(op->H, op->thick, op->z_top, 2 * PI_ * op->freq, khat, pp, rec.data() + size_t(2 * i + 1) * PW_REC);
    }
    da.upload(rec, s);
    farfield_layered(op->mesh, jd.p, op->ne, nrhs, da.p, n, dr.p, s);
  } else {
    std::vector<double> ang(2 * size_t(n));
    for (int i = 0; i < n; ++i) {
      ang[2 * i] = theta[i];
      ang[2 * i + 1] = phi[i];
    }
    da.upload(ang, s);
    farfield(op->mesh, op->k0, jd.p, op->ne, nrhs, da.p, n, dr.p, s);
  }
  SLDM_CUDA(cudaMemcpyAsync(rcs, dr.p, size_t(n) * nrhs * sizeof(double), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  API_END
}

int sldm_farfield(const sldm_op* op, const void* x, int32_t where, const double* theta, const double* phi, int32_t n,
                  double* rcs) {
  return sldm_farfield_n(op, x, 1, where, theta, phi, n, rcs);
}

}  // extern "C"
