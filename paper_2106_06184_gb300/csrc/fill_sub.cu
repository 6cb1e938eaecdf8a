// Good-conductor fill (Sec. II-B: inside highly conductive objects the entries
// need integration that follows the decay of G over a skin depth).  A source
// triangle with an edge longer than 1/|Im k| is bisected through the midpoint
// of its longest edge, recursively, until no child has an edge longer than
// 1/|Im k|, and the 6-point rule runs on each child; the rules are built on the
// host per source.  Touching pairs extract 1/(4 pi R) in closed form (and
// -k^2 R/(8 pi) as well for an unsplit source, as the unsplit kernels do); for
// Kbar the static grad 1/(4 pi R) is extracted as always.  Pairs whose bounding
// spheres are farther apart than 40/|Im k| are dropped (G has decayed below e^-40).
//
// One warp per (test, source) pair: the lanes stride over the 6 x (points of
// the source's rule) (test point, source point) pairs, the lanes 0..5 add the closed forms
// of test point q = lane on touching pairs, the moments are summed with
// shuffles, and lane 0 scatters the 3x3 local block as the unsplit kernels do.
// Everything is FP64; the destination precision is R.
#include <algorithm>
#include <string>
#include <vector>

#include "fill_dev.cuh"

namespace sldm {

constexpr double R8_CUTOFF = 40.0;
constexpr int SUB_MAX_CHILDREN = 4096;  // most children of one split source
constexpr double SPLIT_TIE = 1e-9;      // edges within this relative distance of the longest count as longest

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// (exp(-j k R) - 1)/(4 pi R), Taylor series for |kR| < 0.05
__device__ cd green_smooth1(cd k, double R) {
  const double ax = sqrt(k.r * k.r + k.i * k.i) * R;
  if (ax < 0.05) {
    const cd mjk = {k.i, -k.r};  // -j k
    cd p = mjk, acc = mjk;
    double Rp = 1.0, fact = 1.0;
    for (int n = 2; n <= 11; ++n) {
      p = cmul(p, mjk);
      Rp *= R;
      fact *= n;
      acc.r += p.r * Rp / fact;
      acc.i += p.i * Rp / fact;
    }
    return {acc.r * INV4PI, acc.i * INV4PI};
  }
  double sn, cn;
  sincos(k.r * R, &sn, &cn);
  const double ex = exp(k.i * R);
  return {(ex * cn - 1.0) * INV4PI / R, -ex * sn * INV4PI / R};
}

// G = exp(-j k R)/(4 pi R), from R and 1/R (no division on the FP64 pipe)
__device__ __forceinline__ cd green_full(cd k, double R, double iR) {
  double sn, cn;
  sincos(k.r * R, &sn, &cn);
  const double a = exp(k.i * R) * INV4PI * iR;
  return {a * cn, -a * sn};
}

// g1 of grad G = (r - r') g1 = -(1 + j k R) exp(-j k R)/(4 pi R^3)
__device__ __forceinline__ cd grad_full(cd k, double R, double iR) {
  double sn, cn;
  sincos(k.r * R, &sn, &cn);
  const double a = exp(k.i * R) * INV4PI * (iR * iR * iR);
  const cd e = {a * cn, -a * sn};
  const cd f = {1.0 - k.i * R, k.r * R};  // 1 + j k R
  const cd p = cmul(f, e);
  return {-p.r, -p.i};
}

__device__ __forceinline__ void src_point(const SrcPoint& b, const double ev[3][3], double rp[3]) {
  for (int d = 0; d < 3; ++d) rp[d] = b.x * ev[0][d] + b.y * ev[1][d] + b.z * ev[2][d];
}

__device__ __forceinline__ double bound_radius(const double* c, const double* p0, const double* p1, const double* p2) {
  double r = 0.0;
  const double* P[3] = {p0, p1, p2};
  for (int i = 0; i < 3; ++i) {
    const double dx = P[i][0] - c[0], dy = P[i][1] - c[1], dz = P[i][2] - c[2];
    r = fmax(r, sqrt(dx * dx + dy * dy + dz * dz));
  }
  return r;
}

// ---------------------------------------------------------------- L^A, L^phi
template <class R>
__global__ void __launch_bounds__(256) fill_L_split(LTask tk, const int32_t* __restrict__ soff,
                                                    const SrcPoint* __restrict__ spts,
                                                    const double* __restrict__ geo, const double* __restrict__ xyz,
                                                    const int32_t* __restrict__ tri, const int32_t* __restrict__ tri_edge) {
  const int64_t pair = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pair >= int64_t(tk.ntest) * tk.nsrc) return;  // whole warps
  const int t = tk.t0 + int(pair / tk.nsrc), s = tk.s0 + int(pair % tk.nsrc);
  const double* gt = geo + size_t(t) * GEO_STRIDE;
  const double* gs = geo + size_t(s) * GEO_STRIDE;
  const int32_t sv[3] = {tri[3 * s], tri[3 * s + 1], tri[3 * s + 2]};
  bool touch = false;
  for (int i = 0; i < 3; ++i) {
    const int32_t tv = tri[3 * t + i];
    touch |= (tv == sv[0]) | (tv == sv[1]) | (tv == sv[2]);
  }
  const double* ps[3] = {xyz + 3 * sv[0], xyz + 3 * sv[1], xyz + 3 * sv[2]};
  if (!touch) {
    const double rt = bound_radius(gt + GEO_C, xyz + 3 * tri[3 * t], xyz + 3 * tri[3 * t + 1], xyz + 3 * tri[3 * t + 2]);
    const double rs = bound_radius(gs + GEO_C, ps[0], ps[1], ps[2]);
    const double dx = gt[GEO_C] - gs[GEO_C], dy = gt[GEO_C + 1] - gs[GEO_C + 1], dz = gt[GEO_C + 2] - gs[GEO_C + 2];
    if (fabs(tk.ki) * (sqrt(dx * dx + dy * dy + dz * dz) - rt - rs) > R8_CUTOFF) return;
  }
  const SrcPoint* rule = spts + soff[s - tk.s0];
  const int nu = soff[s - tk.s0 + 1] - soff[s - tk.s0];
  const bool split = nu > 6;
  const double As = gs[GEO_A];
  double ev[3][3], dc[3];
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) ev[i][d] = ps[i][d] - gs[GEO_C + d];
  for (int d = 0; d < 3; ++d) dc[d] = gt[GEO_C + d] - gs[GEO_C + d];
  const cd k = {tk.kr, tk.ki};
  // m: M0 (0,1), Mq (2..7), Ms (8..13), Mqs (14,15)
  double m[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) m[i] = 0.0;
  // unit u = (source point u / 6, test point u % 6): 36 units even when unsplit
  for (int u = lane; u < 6 * nu; u += 32) {
    const int pnt = u / 6, q = u - 6 * pnt;
    const SrcPoint sp = rule[pnt];
    double rp[3];
    src_point(sp, ev, rp);
    const double ws = As * sp.w;
    const double* rq = gt + GEO_RHO + 3 * q;
    const double D0 = dc[0] + rq[0] - rp[0], D1 = dc[1] + rq[1] - rp[1], D2 = dc[2] + rq[2] - rp[2];
    const double r2 = D0 * D0 + D1 * D1 + D2 * D2;
    const double iR = rsqrt(r2), Rr = r2 * iR;
    cd g = touch ? (split ? green_smooth1(k, sqrt(r2)) : green_smooth(k, sqrt(r2))) : green_full(k, Rr, iR);
    const double w = gt[GEO_W + q] * ws;
    g.r *= w;
    g.i *= w;
    const double qs = rq[0] * rp[0] + rq[1] * rp[1] + rq[2] * rp[2];
    m[0] += g.r;
    m[1] += g.i;
    for (int d = 0; d < 3; ++d) {
      m[2 + 2 * d] += g.r * rq[d];
      m[3 + 2 * d] += g.i * rq[d];
      m[8 + 2 * d] += g.r * rp[d];
      m[9 + 2 * d] += g.i * rp[d];
    }
    m[14] += g.r * qs;
    m[15] += g.i * qs;
  }
  if (touch && lane < 6) {
    const int q = lane;
    const double* rq = gt + GEO_RHO + 3 * q;
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = gt[GEO_C + d] + rq[d];
    Pot P;
    potentials(r, ps[0], ps[1], ps[2], P);
    const cd k2 = cmul(k, k);
    const double two = split ? 0.0 : 1.0;  // the k^2 R term is extracted only when unsplit
    cd A = {INV4PI * P.inv_r - two * k2.r * 0.5 * INV4PI * P.r, -two * k2.i * 0.5 * INV4PI * P.r};
    cd Bv[3];
    for (int d = 0; d < 3; ++d) {
      const double off = P.rho[d] - gs[GEO_C + d];
      const double s1 = P.por[d] + off * P.inv_r;
      const double sR = P.pr[d] + off * P.r;
      Bv[d] = {INV4PI * s1 - two * k2.r * 0.5 * INV4PI * sR, -two * k2.i * 0.5 * INV4PI * sR};
    }
    const double w = gt[GEO_W + q];
    m[0] += w * A.r;
    m[1] += w * A.i;
    for (int d = 0; d < 3; ++d) {
      m[2 + 2 * d] += w * A.r * rq[d];
      m[3 + 2 * d] += w * A.i * rq[d];
      m[8 + 2 * d] += w * Bv[d].r;
      m[9 + 2 * d] += w * Bv[d].i;
      m[14] += w * rq[d] * Bv[d].r;
      m[15] += w * rq[d] * Bv[d].i;
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) m[i] = warp_sum(m[i]);
  if (lane != 0) return;
  const cd m0 = {m[0], m[1]}, mqs = {m[14], m[15]};
  cd mq[3], ms[3];
  for (int d = 0; d < 3; ++d) {
    mq[d] = {m[2 + 2 * d], m[3 + 2 * d]};
    ms[d] = {m[8 + 2 * d], m[9 + 2 * d]};
  }
  if (tk.A) {
    for (int i = 0; i < 3; ++i) {
      const double* a = gt + GEO_AV + 3 * i;
      for (int j = 0; j < 3; ++j) {
        const double* b = gs + GEO_AV + 3 * j;
        const double ab = a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
        cd v = mqs;
        for (int d = 0; d < 3; ++d) {
          v.r += a[d] * ms[d].r + b[d] * mq[d].r;
          v.i += a[d] * ms[d].i + b[d] * mq[d].i;
        }
        v.r += ab * m0.r;
        v.i += ab * m0.i;
        const double sc = gt[GEO_SIG + i] * gs[GEO_SIG + j];
        const cd out = cmul({v.r * sc, v.i * sc}, {tk.sAr, tk.sAi});
        add_d<R>(tk.A, int64_t(tri_edge[3 * t + i] - tk.e_row0) * tk.ldA + (tri_edge[3 * s + j] - tk.e_col0), out.r, out.i);
      }
    }
  }
  if (tk.P) {
    const double sc = 1.0 / (gt[GEO_A] * gs[GEO_A]);
    const cd out = cmul({m0.r * sc, m0.i * sc}, {tk.sPr, tk.sPi});
    M<R>::store(tk.P, int64_t(t - tk.t_row0) * tk.ldP + (s - tk.t_col0), out.r, out.i);
  }
}

// ---------------------------------------------------------------- Kbar (primal test x barycentric child)
template <class R>
__global__ void __launch_bounds__(256) fill_K_split(KTask tk, const int32_t* __restrict__ soff,
                                                    const SrcPoint* __restrict__ spts,
                                                    const double* __restrict__ geo,
                                                    const double* __restrict__ bgeo, const double* __restrict__ xyz,
                                                    const int32_t* __restrict__ tri, const int32_t* __restrict__ tri_edge,
                                                    const int32_t* __restrict__ btri_edge) {
  const int64_t pair = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (pair >= int64_t(tk.ntest) * tk.nsrc) return;
  const int t = tk.t0 + int(pair / tk.nsrc), cg = tk.c0 + int(pair % tk.nsrc);
  const int par = cg / 6, kk = cg % 6, pp = kk / 2;
  if (par == t) return;  // child of the test triangle: coplanar, Kbar = 0
  const int32_t cvx = tri[3 * par + ((kk & 1) ? (pp + 1) % 3 : pp)];  // child's primal vertex
  const int32_t ce = tri_edge[3 * par + (pp + 2) % 3];                 // edge of the child's midpoint
  bool touch = false;
  for (int i = 0; i < 3; ++i) touch |= (tri[3 * t + i] == cvx) | (tri_edge[3 * t + i] == ce);
  const double* gt = geo + size_t(t) * GEO_STRIDE;
  const double* gs = bgeo + size_t(cg) * GEO_STRIDE;
  // child vertices rebuilt from the parent: (a, m_ab, g) (m_ab, b, g) (b, m_bc, g) (m_bc, c, g) (c, m_ca, g) (m_ca, a, g)
  const double* a = xyz + 3 * tri[3 * par];
  const double* b = xyz + 3 * tri[3 * par + 1];
  const double* c = xyz + 3 * tri[3 * par + 2];
  double V[7][3];
  for (int d = 0; d < 3; ++d) {
    V[0][d] = a[d]; V[1][d] = b[d]; V[2][d] = c[d];
    V[3][d] = 0.5 * (a[d] + b[d]); V[4][d] = 0.5 * (b[d] + c[d]); V[5][d] = 0.5 * (c[d] + a[d]);
    V[6][d] = (a[d] + b[d] + c[d]) / 3.0;
  }
  const int cvt[6][3] = {{0, 3, 6}, {3, 1, 6}, {1, 4, 6}, {4, 2, 6}, {2, 5, 6}, {5, 0, 6}};
  const double* ps[3] = {V[cvt[kk][0]], V[cvt[kk][1]], V[cvt[kk][2]]};
  if (!touch) {
    const double rt = bound_radius(gt + GEO_C, xyz + 3 * tri[3 * t], xyz + 3 * tri[3 * t + 1], xyz + 3 * tri[3 * t + 2]);
    const double rs = bound_radius(gs + GEO_C, ps[0], ps[1], ps[2]);
    const double dx = gt[GEO_C] - gs[GEO_C], dy = gt[GEO_C + 1] - gs[GEO_C + 1], dz = gt[GEO_C + 2] - gs[GEO_C + 2];
    if (fabs(tk.ki) * (sqrt(dx * dx + dy * dy + dz * dz) - rt - rs) > R8_CUTOFF) return;
  }
  const SrcPoint* rule = spts + soff[cg - tk.c0];
  const int nu = soff[cg - tk.c0 + 1] - soff[cg - tk.c0];
  const double As = gs[GEO_A];
  double ev[3][3], dc[3];
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) ev[i][d] = ps[i][d] - gs[GEO_C + d];
  for (int d = 0; d < 3; ++d) dc[d] = gt[GEO_C + d] - gs[GEO_C + d];
  const cd k = {tk.kr, tk.ki};
  // m: P1 (0,1), P2 (2..7), X (8..13), S (14..19)
  double m[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = 0.0;
  // unit u = (source point u / 6, test point u % 6)
  for (int u = lane; u < 6 * nu; u += 32) {
    const int pnt = u / 6, q = u - 6 * pnt;
    const SrcPoint sp = rule[pnt];
    double rp[3];
    src_point(sp, ev, rp);
    const double ws = As * sp.w;
    const double* rq = gt + GEO_RHO + 3 * q;
    const double D[3] = {dc[0] + rq[0] - rp[0], dc[1] + rq[1] - rp[1], dc[2] + rq[2] - rp[2]};
    const double r2 = D[0] * D[0] + D[1] * D[1] + D[2] * D[2];
    const double iR = rsqrt(r2), Rr = r2 * iR;
    cd g1 = touch ? grad_smooth(k, sqrt(r2)) : grad_full(k, Rr, iR);
    const double w = gt[GEO_W + q] * ws;
    g1.r *= w;
    g1.i *= w;
    const double cr[3] = {D[1] * rp[2] - D[2] * rp[1], D[2] * rp[0] - D[0] * rp[2], D[0] * rp[1] - D[1] * rp[0]};
    const double xq[3] = {rq[1] * D[2] - rq[2] * D[1], rq[2] * D[0] - rq[0] * D[2], rq[0] * D[1] - rq[1] * D[0]};
    const double p1 = rq[0] * cr[0] + rq[1] * cr[1] + rq[2] * cr[2];
    m[0] += g1.r * p1;
    m[1] += g1.i * p1;
    for (int d = 0; d < 3; ++d) {
      m[2 + 2 * d] += g1.r * cr[d];
      m[3 + 2 * d] += g1.i * cr[d];
      m[8 + 2 * d] += g1.r * xq[d];
      m[9 + 2 * d] += g1.i * xq[d];
      m[14 + 2 * d] += g1.r * D[d];
      m[15 + 2 * d] += g1.i * D[d];
    }
  }
  if (touch && lane < 6) {
    // static part: V_s = int grad 1/(4 pi R) dS', U_s = V_s x (r - c')
    const int q = lane;
    const double* rq = gt + GEO_RHO + 3 * q;
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = gt[GEO_C + d] + rq[d];
    Pot P;
    potentials(r, ps[0], ps[1], ps[2], P);
    double vs[3], rc[3];
    for (int d = 0; d < 3; ++d) {
      vs[d] = INV4PI * P.grad[d];
      rc[d] = r[d] - gs[GEO_C + d];
    }
    const double us[3] = {vs[1] * rc[2] - vs[2] * rc[1], vs[2] * rc[0] - vs[0] * rc[2], vs[0] * rc[1] - vs[1] * rc[0]};
    const double w = gt[GEO_W + q];
    m[0] += w * (rq[0] * us[0] + rq[1] * us[1] + rq[2] * us[2]);
    const double xq[3] = {rq[1] * vs[2] - rq[2] * vs[1], rq[2] * vs[0] - rq[0] * vs[2], rq[0] * vs[1] - rq[1] * vs[0]};
    for (int d = 0; d < 3; ++d) {
      m[2 + 2 * d] += w * us[d];
      m[8 + 2 * d] += w * xq[d];
      m[14 + 2 * d] += w * vs[d];
    }
  }
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = warp_sum(m[i]);
  if (lane != 0) return;
  const cd P1 = {m[0], m[1]};
  cd P2[3], X[3], S[3];
  for (int d = 0; d < 3; ++d) {
    P2[d] = {m[2 + 2 * d], m[3 + 2 * d]};
    X[d] = {m[8 + 2 * d], m[9 + 2 * d]};
    S[d] = {m[14 + 2 * d], m[15 + 2 * d]};
  }
  for (int i = 0; i < 3; ++i) {
    const double* av = gt + GEO_AV + 3 * i;
    cd base = P1;
    for (int d = 0; d < 3; ++d) {
      base.r += av[d] * P2[d].r;
      base.i += av[d] * P2[d].i;
    }
    const cd axs[3] = {{av[1] * S[2].r - av[2] * S[1].r, av[1] * S[2].i - av[2] * S[1].i},
                       {av[2] * S[0].r - av[0] * S[2].r, av[2] * S[0].i - av[0] * S[2].i},
                       {av[0] * S[1].r - av[1] * S[0].r, av[0] * S[1].i - av[1] * S[0].i}};
    for (int j = 0; j < 3; ++j) {
      const double* bv = gs + GEO_AV + 3 * j;
      cd v = base;
      for (int d = 0; d < 3; ++d) {
        v.r += bv[d] * (X[d].r + axs[d].r);
        v.i += bv[d] * (X[d].i + axs[d].i);
      }
      const double sc = gt[GEO_SIG + i] * gs[GEO_SIG + j];
      add_d<R>(tk.Kb, int64_t(tri_edge[3 * t + i] - tk.e_row0) * tk.ld + (btri_edge[3 * cg + j] - tk.b_col0), v.r * sc,
               v.i * sc);
    }
  }
}

// ---------------------------------------------------------------- host side
static const double kBary[6][3] = {
    {0.108103018168070, 0.445948490915965, 0.445948490915965}, {0.445948490915965, 0.108103018168070, 0.445948490915965},
    {0.445948490915965, 0.445948490915965, 0.108103018168070}, {0.816847572980459, 0.091576213509771, 0.091576213509771},
    {0.091576213509771, 0.816847572980459, 0.091576213509771}, {0.091576213509771, 0.091576213509771, 0.816847572980459}};
static const double kW[6] = {0.223381589678011, 0.223381589678011, 0.223381589678011,
                              0.109951743655322, 0.109951743655322, 0.109951743655322};

static double edge_len(const double* a, const double* b) {
  return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
}

// The source's quadrature appended to `pts`: longest-edge bisection of the
// triangle (p0, p1, p2) until no child has an edge longer than h (edge i joins
// vertices i and i + 1; the first edge within SPLIT_TIE of the longest is cut;
// the child holding the cut edge's first vertex is refined first), then the
// 6-point rule on each child.
struct Child {
  double B[3][3];  // barycentric coordinates of the child's vertices
  double f;        // area fraction
};
static void append_rule(const double* p0, const double* p1, const double* p2, double h, std::vector<SrcPoint>& pts) {
  const double* P[3] = {p0, p1, p2};
  std::vector<Child> todo(1), done;
  todo[0] = Child{{{1, 0, 0}, {0, 1, 0}, {0, 0, 1}}, 1.0};
  while (!todo.empty()) {
    const Child c = todo.back();
    todo.pop_back();
    double X[3][3];
    for (int v = 0; v < 3; ++v)
      for (int d = 0; d < 3; ++d) X[v][d] = c.B[v][0] * P[0][d] + c.B[v][1] * P[1][d] + c.B[v][2] * P[2][d];
    const double L[3] = {edge_len(X[0], X[1]), edge_len(X[1], X[2]), edge_len(X[2], X[0])};
    const double Lmax = std::max(L[0], std::max(L[1], L[2]));
    if (!(Lmax > h)) {
      done.push_back(c);
      continue;
    }
    int i = 0;
    while (!(L[i] >= (1.0 - SPLIT_TIE) * Lmax)) ++i;
    const double* a = c.B[i];
    const double* b = c.B[(i + 1) % 3];
    const double* cc = c.B[(i + 2) % 3];
    Child c1, c2;
    for (int d = 0; d < 3; ++d) {
      const double m = 0.5 * (a[d] + b[d]);
      c1.B[0][d] = m; c1.B[1][d] = b[d]; c1.B[2][d] = cc[d];
      c2.B[0][d] = a[d]; c2.B[1][d] = m; c2.B[2][d] = cc[d];
    }
    c1.f = c2.f = 0.5 * c.f;
    todo.push_back(c1);
    todo.push_back(c2);
    SLDM_REQUIRE(done.size() + todo.size() <= size_t(SUB_MAX_CHILDREN), SLDM_ENOTSUP,
                 "source triangle too large for the skin depth: more than " + std::to_string(SUB_MAX_CHILDREN) +
                     " children");
  }
  for (const Child& c : done)
    for (int j = 0; j < 6; ++j) {
      double b[3] = {0, 0, 0};
      for (int v = 0; v < 3; ++v)
        for (int d = 0; d < 3; ++d) b[d] += kBary[j][v] * c.B[v][d];
      pts.push_back(SrcPoint{b[0], b[1], b[2], c.f * kW[j]});
    }
}

static double longest_edge(const double* p0, const double* p1, const double* p2) {
  return std::max(edge_len(p0, p2), std::max(edge_len(p1, p0), edge_len(p2, p1)));
}

template <class VertexFn>
static SplitRules make_rules(int nsrc, double ki, VertexFn vertices) {
  SplitRules R;
  const double aki = std::fabs(ki);
  for (int i = 0; i < nsrc && !R.split; ++i) {
    const double* p[3];
    double store[3][3];
    vertices(i, p, store);
    R.split = aki * longest_edge(p[0], p[1], p[2]) > 1.0;
  }
  if (!R.split) return R;
  const double h = 1.0 / aki;
  R.off.reserve(size_t(nsrc) + 1);
  for (int i = 0; i < nsrc; ++i) {
    R.off.push_back(int32_t(R.pts.size()));
    const double* p[3];
    double store[3][3];
    vertices(i, p, store);
    append_rule(p[0], p[1], p[2], h, R.pts);
  }
  R.off.push_back(int32_t(R.pts.size()));
  return R;
}

SplitRules split_rules_L(const HostMesh& h, const LTask& tk) {
  return make_rules(tk.nsrc, tk.ki, [&](int i, const double* p[3], double (*)[3]) {
    const int s = tk.s0 + i;
    for (int v = 0; v < 3; ++v) p[v] = &h.xyz[3 * size_t(h.tri[3 * s + v])];
  });
}

SplitRules split_rules_K(const HostMesh& h, const KTask& tk) {
  static const int cvt[6][3] = {{0, 3, 6}, {3, 1, 6}, {1, 4, 6}, {4, 2, 6}, {2, 5, 6}, {5, 0, 6}};
  return make_rules(tk.nsrc, tk.ki, [&](int i, const double* p[3], double (*store)[3]) {
    const int cg = tk.c0 + i, par = cg / 6, kk = cg % 6;
    const double* a = &h.xyz[3 * size_t(h.tri[3 * par])];
    const double* b = &h.xyz[3 * size_t(h.tri[3 * par + 1])];
    const double* c = &h.xyz[3 * size_t(h.tri[3 * par + 2])];
    double V[7][3];
    for (int d = 0; d < 3; ++d) {
      V[0][d] = a[d]; V[1][d] = b[d]; V[2][d] = c[d];
      V[3][d] = 0.5 * (a[d] + b[d]); V[4][d] = 0.5 * (b[d] + c[d]); V[5][d] = 0.5 * (c[d] + a[d]);
      V[6][d] = (a[d] + b[d] + c[d]) / 3.0;
    }
    for (int v = 0; v < 3; ++v) {
      for (int d = 0; d < 3; ++d) store[v][d] = V[cvt[kk][v]][d];
      p[v] = store[v];
    }
  });
}

template <class R>
void fill_L_split_task(const sldm_mesh* m, const LTask& tk, const SplitRules& rules, cudaStream_t s) {
  DBuf<int32_t> doff;
  DBuf<SrcPoint> dpts;
  doff.upload(rules.off, s);
  dpts.upload(rules.pts, s);
  const int64_t threads = int64_t(tk.ntest) * tk.nsrc * 32;
  const DevMesh& d = m->d;
  {
    ScopedTimer tm("fill_L_split", s);
    fill_L_split<R><<<unsigned((threads + 255) / 256), 256, 0, s>>>(tk, doff.p, dpts.p, d.geo.p, d.xyz.p, d.tri.p,
                                                                   d.tri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaStreamSynchronize(s));
}

template <class R>
void fill_K_split_task(const sldm_mesh* m, const KTask& tk, const SplitRules& rules, cudaStream_t s) {
  DBuf<int32_t> doff;
  DBuf<SrcPoint> dpts;
  doff.upload(rules.off, s);
  dpts.upload(rules.pts, s);
  const int64_t threads = int64_t(tk.ntest) * tk.nsrc * 32;
  const DevMesh& d = m->d;
  {
    ScopedTimer tm("fill_K_split", s);
    fill_K_split<R><<<unsigned((threads + 255) / 256), 256, 0, s>>>(tk, doff.p, dpts.p, d.geo.p, d.bgeo.p, d.xyz.p, d.tri.p,
                                                                   d.tri_edge.p, d.btri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaStreamSynchronize(s));
}

template void fill_L_split_task<float>(const sldm_mesh*, const LTask&, const SplitRules&, cudaStream_t);
template void fill_L_split_task<double>(const sldm_mesh*, const LTask&, const SplitRules&, cudaStream_t);
template void fill_K_split_task<float>(const sldm_mesh*, const KTask&, const SplitRules&, cudaStream_t);
template void fill_K_split_task<double>(const sldm_mesh*, const KTask&, const SplitRules&, cudaStream_t);

}  // namespace sldm
