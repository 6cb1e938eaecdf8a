// Triangle-pair Gauss-quadrature fill of the SLDM operators (Sec. II-B, II-C):
//   L^A[m,n]   = int f_m . int f_n G        (RWG x RWG)           Eq. opLAhgf
//   L^phi[p,q] = int int h_p h_q G          (pulse x pulse)       Eq. opLphihgf
//   Kbar[m,k]  = int f_m . PV int grad G x g_k   (RWG x barycentric RWG; the BC
//                functions are sums of g_k, contracted afterwards)  Eq. opKhgf
// with G = exp(-j k R)/(4 pi R) (Eq. hgf), 6-point Dunavant rules on both
// triangles, and singularity extraction on touching pairs computed in FP64.
//
// GPU design: every pair is reduced to a handful of complex "moments" in
// triangle-local coordinates (r = c + rho), so that the 3x3 RWG combinations
// and the absolute coordinates never enter the inner loop.  One thread owns a
// source triangle (coalesced SoA record), a CTA walks a tile of test triangles
// held in shared memory, and the 3x3 results are scattered with atomics
// (each edge-pair entry gets four triangle-pair contributions).
#include <algorithm>
#include <cmath>
#include <mutex>
#include <new>

#include "fill_dev.cuh"

namespace sldm {

// ---------------------------------------------------------------- geometry
// Writes a GEO_STRIDE record for a triangle with vertices p0, p1, p2 and edge
// signs s (s_i for the edge opposite vertex i).
__device__ void write_geo(double* g, const double* p0, const double* p1, const double* p2, const double s[3]) {
  double c[3], u[3], w[3], cr[3];
  for (int d = 0; d < 3; ++d) {
    c[d] = (p0[d] + p1[d] + p2[d]) / 3.0;
    u[d] = p1[d] - p0[d];
    w[d] = p2[d] - p0[d];
  }
  cr[0] = u[1] * w[2] - u[2] * w[1];
  cr[1] = u[2] * w[0] - u[0] * w[2];
  cr[2] = u[0] * w[1] - u[1] * w[0];
  double n2 = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  double A = 0.5 * n2;
  for (int d = 0; d < 3; ++d) {
    g[GEO_C + d] = c[d];
    g[GEO_N + d] = cr[d] / n2;
  }
  g[GEO_A] = A;
  const double* P[3] = {p0, p1, p2};
  for (int q = 0; q < 6; ++q) {
    for (int d = 0; d < 3; ++d) {
      double r = c_bary[q][0] * p0[d] + c_bary[q][1] * p1[d] + c_bary[q][2] * p2[d];
      g[GEO_RHO + 3 * q + d] = r - c[d];
    }
    g[GEO_W + q] = c_w[q] * A;
  }
  for (int i = 0; i < 3; ++i) {
    for (int d = 0; d < 3; ++d) g[GEO_AV + 3 * i + d] = c[d] - P[i][d];
    g[GEO_SIG + i] = s[i] / (2.0 * A);
  }
}

__global__ void geometry_kernel(int nt, const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                                const int32_t* __restrict__ tri_edge, const int8_t* __restrict__ tri_sign,
                                const int8_t* __restrict__ btri_sign, int64_t nv, double* geo, double* bgeo) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const double* a = xyz + 3 * tri[3 * t];
  const double* b = xyz + 3 * tri[3 * t + 1];
  const double* c = xyz + 3 * tri[3 * t + 2];
  double s[3] = {double(tri_sign[3 * t]), double(tri_sign[3 * t + 1]), double(tri_sign[3 * t + 2])};
  write_geo(geo + size_t(t) * GEO_STRIDE, a, b, c, s);
  double mab[3], mbc[3], mca[3], g[3];
  for (int d = 0; d < 3; ++d) {
    mab[d] = 0.5 * (a[d] + b[d]);
    mbc[d] = 0.5 * (b[d] + c[d]);
    mca[d] = 0.5 * (c[d] + a[d]);
    g[d] = (a[d] + b[d] + c[d]) / 3.0;
  }
  // children: (a, m_ab, g) (m_ab, b, g) (b, m_bc, g) (m_bc, c, g) (c, m_ca, g) (m_ca, a, g)
  const double* ch[6][3] = {{a, mab, g}, {mab, b, g}, {b, mbc, g}, {mbc, c, g}, {c, mca, g}, {mca, a, g}};
  for (int k = 0; k < 6; ++k) {
    int cc = 6 * t + k;
    double sb[3] = {double(btri_sign[3 * cc]), double(btri_sign[3 * cc + 1]), double(btri_sign[3 * cc + 2])};
    write_geo(bgeo + size_t(cc) * GEO_STRIDE, ch[k][0], ch[k][1], ch[k][2], sb);
  }
}

void geometry(const HostMesh& hm, DevMesh& dm, cudaStream_t s) {
  dm.geo.alloc(size_t(hm.nt) * GEO_STRIDE);
  dm.bgeo.alloc(size_t(hm.nt) * 6 * GEO_STRIDE);
  int nt = int(hm.nt);
  geometry_kernel<<<(nt + 127) / 128, 128, 0, s>>>(nt, dm.xyz.p, dm.tri.p, dm.tri_edge.p, dm.tri_sign.p,
                                                   dm.btri_sign.p, hm.nv, dm.geo.p, dm.bgeo.p), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- bulk L kernel
constexpr int TILE_SRC = 128;  // source triangles per CTA (one per thread)
constexpr int TILE_TEST = 8;   // test triangles per CTA (FP64 fills)
// Test triangles per CTA: each thread converts its source record to the fill's
// precision once per CTA, so the FP32 fills take 32 test triangles to keep those
// conversions (on the narrow FP64 pipe of this part) off the per-pair cost.
template <class R>
constexpr int tile_test() {
  return sizeof(R) == 4 ? 32 : TILE_TEST;
}

struct TileRef {
  int32_t task, test0, src0, pad;
};

// Centroids as hi + lo in the fill's precision (for FP32: two floats, c to ~2^-48),
// so the centroid difference of a pair, (hi - hi') + (lo - lo'), is formed to the
// fill's precision relative to the distance without FP64 operations in the loop.
template <class R>
struct TestRec {
  R rho[18], W[6], av[9], sig[3];
  R chi[3], clo[3];
  R invA;
  int32_t v[3], e[3];
};
template <class R>
__device__ __forceinline__ void split_hl(double v, R& hi, R& lo) {
  hi = R(v);
  lo = R(v - double(hi));
}

template <class R>
__global__ void __launch_bounds__(TILE_SRC, sizeof(R) == 4 ? 5 : 1) fill_L_bulk(const LTask* __restrict__ tasks, const TileRef* __restrict__ tiles,
                                                        const double* __restrict__ geo, const int32_t* __restrict__ tri,
                                                        const int32_t* __restrict__ tri_edge) {
  __shared__ TestRec<R> T[tile_test<R>()];
  const TileRef tile = tiles[blockIdx.x];
  const LTask tk = tasks[tile.task];
  // load the test tile
  for (int idx = threadIdx.x; idx < tile_test<R>(); idx += blockDim.x) {
    int t = tile.test0 + idx;
    if (t < tk.ntest) {
      int tg = tk.t0 + t;
      const double* g = geo + size_t(tg) * GEO_STRIDE;
      for (int d = 0; d < 18; ++d) T[idx].rho[d] = R(g[GEO_RHO + d]);
      for (int d = 0; d < 6; ++d) T[idx].W[d] = R(g[GEO_W + d]);
      for (int d = 0; d < 9; ++d) T[idx].av[d] = R(g[GEO_AV + d]);
      for (int d = 0; d < 3; ++d) {
        T[idx].sig[d] = R(g[GEO_SIG + d]);
        split_hl(g[GEO_C + d], T[idx].chi[d], T[idx].clo[d]);
        T[idx].v[d] = tri[3 * tg + d];
        T[idx].e[d] = tri_edge[3 * tg + d];
      }
      T[idx].invA = R(1.0 / g[GEO_A]);
    }
  }
  __syncthreads();
  const int s = tile.src0 + threadIdx.x;
  if (s >= tk.nsrc) return;
  const int sg = tk.s0 + s;
  const double* gs = geo + size_t(sg) * GEO_STRIDE;
  R rs[18], Ws[6], bv[9], sg_[3], cshi[3], cslo[3];
#pragma unroll
  for (int d = 0; d < 18; ++d) rs[d] = R(gs[GEO_RHO + d]);
#pragma unroll
  for (int d = 0; d < 6; ++d) Ws[d] = R(gs[GEO_W + d]);
#pragma unroll
  for (int d = 0; d < 9; ++d) bv[d] = R(gs[GEO_AV + d]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sg_[d] = R(gs[GEO_SIG + d]);
    split_hl(gs[GEO_C + d], cshi[d], cslo[d]);
  }
  const R invAs = R(1.0 / gs[GEO_A]);
  const int32_t sv0 = tri[3 * sg], sv1 = tri[3 * sg + 1], sv2 = tri[3 * sg + 2];
  const int32_t se[3] = {tri_edge[3 * sg], tri_edge[3 * sg + 1], tri_edge[3 * sg + 2]};
  const R kr = R(tk.kr), ki = R(tk.ki);
#pragma unroll
  for (int k = 0; k < 6; ++k) Ws[k] *= R(INV4PI);  // 1/(4 pi) of G folded into the source weights
  const R sAr = R(tk.sAr), sAi = R(tk.sAi), sPr = R(tk.sPr), sPi = R(tk.sPi);

  for (int tt = 0; tt < tile_test<R>(); ++tt) {
    if (tile.test0 + tt >= tk.ntest) break;
    const TestRec<R>& X = T[tt];
    // touching pairs (sharing a vertex) are computed by the FP64 extraction kernel
    bool touch = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) touch |= (X.v[i] == sv0) | (X.v[i] == sv1) | (X.v[i] == sv2);
    if (touch) continue;
    const R dc0 = (X.chi[0] - cshi[0]) + (X.clo[0] - cslo[0]);
    const R dc1 = (X.chi[1] - cshi[1]) + (X.clo[1] - cslo[1]);
    const R dc2 = (X.chi[2] - cshi[2]) + (X.clo[2] - cslo[2]);
    R m0r = 0, m0i = 0, mqr[3] = {0, 0, 0}, mqi[3] = {0, 0, 0}, msr[3] = {0, 0, 0}, msi[3] = {0, 0, 0};
    R mqsr = 0, mqsi = 0;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const R px = dc0 + X.rho[3 * q], py = dc1 + X.rho[3 * q + 1], pz = dc2 + X.rho[3 * q + 2];
      R ar = 0, ai = 0, br[3] = {0, 0, 0}, bi[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const R dx = px - rs[3 * k], dy = py - rs[3 * k + 1], dz = pz - rs[3 * k + 2];
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R ir = M<R>::rsqrt_(r2);
        const R Rr = r2 * ir;
        R sn, cn;
        M<R>::sincos_(kr * Rr, &sn, &cn);
        const R amp = (ki != R(0) ? M<R>::exp_(ki * Rr) : R(1)) * ir * Ws[k];
        const R gr = amp * cn, gi = -amp * sn;
        ar += gr;
        ai += gi;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          br[d] += gr * rs[3 * k + d];
          bi[d] += gi * rs[3 * k + d];
        }
      }
      const R w = X.W[q];
      m0r += w * ar;
      m0i += w * ai;
      R dotr = 0, doti = 0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        const R rq = X.rho[3 * q + d];
        mqr[d] += w * ar * rq;
        mqi[d] += w * ai * rq;
        msr[d] += w * br[d];
        msi[d] += w * bi[d];
        dotr += rq * br[d];
        doti += rq * bi[d];
      }
      mqsr += w * dotr;
      mqsi += w * doti;
    }
    // local RWG x RWG: sig_i sig_j [Mqs + a_i.Ms + b_j.Mq + (a_i.b_j) M0]
    if (tk.A) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R ax = X.av[3 * i], ay = X.av[3 * i + 1], az = X.av[3 * i + 2];
        const R ams_r = ax * msr[0] + ay * msr[1] + az * msr[2];
        const R ams_i = ax * msi[0] + ay * msi[1] + az * msi[2];
        const int64_t row = int64_t(X.e[i] - tk.e_row0) * tk.ldA;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
          const R bx = bv[3 * j], by = bv[3 * j + 1], bz = bv[3 * j + 2];
          const R ab = ax * bx + ay * by + az * bz;
          R vr = mqsr + ams_r + bx * mqr[0] + by * mqr[1] + bz * mqr[2] + ab * m0r;
          R vi = mqsi + ams_i + bx * mqi[0] + by * mqi[1] + bz * mqi[2] + ab * m0i;
          const R sc = X.sig[i] * sg_[j];
          vr *= sc;
          vi *= sc;
          M<R>::add(tk.A, row + (se[j] - tk.e_col0), vr * sAr - vi * sAi, vr * sAi + vi * sAr);
        }
      }
    }
    if (tk.P) {
      const R sc = X.invA * invAs;
      const R vr = m0r * sc, vi = m0i * sc;
      const int t = tile.test0 + tt;
      M<R>::store_r(tk.P, int64_t(t + tk.t0 - tk.t_row0) * tk.ldP + (sg - tk.t_col0), vr * sPr - vi * sPi,
                    vr * sPi + vi * sPr);
    }
  }
}

// ---------------------------------------------------------------- FP64 touching L pairs
// Eight lanes per pair: lane q < 6 takes outer point q (closed forms + 6-point
// remainder), the pair's moments are summed with shuffles inside the group,
// and lane 0 scatters the 3x3 block.  One launch serves every task: a pair
// belongs to the task of its object (obj_task), or to none.

template <class R>
__global__ void fill_L_touch(const LTask* __restrict__ tasks, const int32_t* __restrict__ obj_task,
                             const int32_t* __restrict__ tri_obj, const int32_t* __restrict__ pa,
                             const int32_t* __restrict__ pb, int npairs, const double* __restrict__ geo,
                             const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                             const int32_t* __restrict__ tri_edge) {
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int p = int(gt >> 3), q = int(gt & 7);
  int task = -1, t = 0, s = 0;
  if (p < npairs) {
    t = pa[p];
    s = pb[p];
    task = obj_task[tri_obj[t]];
  }
  const bool act = task >= 0 && q < 6;
  LTask tk;
  if (task >= 0) tk = tasks[task];
  double m[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) m[i] = 0.0;
  const double* gt_ = geo + size_t(t) * GEO_STRIDE;
  const double* gs = geo + size_t(s) * GEO_STRIDE;
  if (act) {
    const cd k = {tk.kr, tk.ki};
    const cd k2 = cmul(k, k);
    double r[3];
    for (int d = 0; d < 3; ++d) r[d] = gt_[GEO_C + d] + gt_[GEO_RHO + 3 * q + d];
    cd A = {0, 0}, B[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int j = 0; j < 6; ++j) {
      const double dx = r[0] - gs[GEO_C] - gs[GEO_RHO + 3 * j];
      const double dy = r[1] - gs[GEO_C + 1] - gs[GEO_RHO + 3 * j + 1];
      const double dz = r[2] - gs[GEO_C + 2] - gs[GEO_RHO + 3 * j + 2];
      const cd g = green_smooth(k, sqrt(dx * dx + dy * dy + dz * dz));
      const double w = gs[GEO_W + j];
      A.r += w * g.r;
      A.i += w * g.i;
      for (int d = 0; d < 3; ++d) {
        B[d].r += w * g.r * gs[GEO_RHO + 3 * j + d];
        B[d].i += w * g.i * gs[GEO_RHO + 3 * j + d];
      }
    }
    Pot P;
    potentials(r, xyz + 3 * tri[3 * s], xyz + 3 * tri[3 * s + 1], xyz + 3 * tri[3 * s + 2], P);
    A.r += INV4PI * P.inv_r - k2.r * 0.5 * INV4PI * P.r;
    A.i += -k2.i * 0.5 * INV4PI * P.r;
    for (int d = 0; d < 3; ++d) {
      const double off = P.rho[d] - gs[GEO_C + d];  // (r' - c') = P + (rho - c')
      const double s1 = P.por[d] + off * P.inv_r;
      const double sR = P.pr[d] + off * P.r;
      B[d].r += INV4PI * s1 - k2.r * 0.5 * INV4PI * sR;
      B[d].i += -k2.i * 0.5 * INV4PI * sR;
    }
    const double w = gt_[GEO_W + q];
    m[0] = w * A.r;
    m[1] = w * A.i;
    for (int d = 0; d < 3; ++d) {
      const double rq = gt_[GEO_RHO + 3 * q + d];
      m[2 + 2 * d] = w * A.r * rq;       // Mq
      m[3 + 2 * d] = w * A.i * rq;
      m[8 + 2 * d] = w * B[d].r;         // Ms
      m[9 + 2 * d] = w * B[d].i;
      m[14] += w * rq * B[d].r;          // Mqs
      m[15] += w * rq * B[d].i;
    }
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) m[i] = grp_sum8(m[i]);
  if (task < 0 || q != 0) return;
  const cd m0 = {m[0], m[1]}, mqs = {m[14], m[15]};
  cd mq[3], ms[3];
  for (int d = 0; d < 3; ++d) {
    mq[d] = {m[2 + 2 * d], m[3 + 2 * d]};
    ms[d] = {m[8 + 2 * d], m[9 + 2 * d]};
  }
  if (tk.A) {
    for (int i = 0; i < 3; ++i) {
      const double* a = gt_ + GEO_AV + 3 * i;
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
        const double sc = gt_[GEO_SIG + i] * gs[GEO_SIG + j];
        const cd out = cmul({v.r * sc, v.i * sc}, {tk.sAr, tk.sAi});
        add_d<R>(tk.A, int64_t(tri_edge[3 * t + i] - tk.e_row0) * tk.ldA + (tri_edge[3 * s + j] - tk.e_col0), out.r, out.i);
      }
    }
  }
  if (tk.P) {
    const double sc = 1.0 / (gt_[GEO_A] * gs[GEO_A]);
    const cd out = cmul({m0.r * sc, m0.i * sc}, {tk.sPr, tk.sPi});
    M<R>::store(tk.P, int64_t(t - tk.t_row0) * tk.ldP + (s - tk.t_col0), out.r, out.i);
  }
}

// ---------------------------------------------------------------- bulk Kbar kernel (primal test x child source)
template <class R>
__global__ void __launch_bounds__(TILE_SRC, sizeof(R) == 4 ? 5 : 1) fill_K_bulk(const KTask* __restrict__ tasks, const TileRef* __restrict__ tiles,
                                                        const double* __restrict__ geo, const double* __restrict__ bgeo,
                                                        const int32_t* __restrict__ tri, const int32_t* __restrict__ tri_edge,
                                                        const int32_t* __restrict__ btri_edge) {
  __shared__ TestRec<R> T[tile_test<R>()];
  const TileRef tile = tiles[blockIdx.x];
  const KTask tk = tasks[tile.task];
  for (int idx = threadIdx.x; idx < tile_test<R>(); idx += blockDim.x) {
    int t = tile.test0 + idx;
    if (t < tk.ntest) {
      int tg = tk.t0 + t;
      const double* g = geo + size_t(tg) * GEO_STRIDE;
      for (int d = 0; d < 18; ++d) T[idx].rho[d] = R(g[GEO_RHO + d]);
      for (int d = 0; d < 6; ++d) T[idx].W[d] = R(g[GEO_W + d]);
      for (int d = 0; d < 9; ++d) T[idx].av[d] = R(g[GEO_AV + d]);
      for (int d = 0; d < 3; ++d) {
        T[idx].sig[d] = R(g[GEO_SIG + d]);
        split_hl(g[GEO_C + d], T[idx].chi[d], T[idx].clo[d]);
        T[idx].v[d] = tri[3 * tg + d];
        T[idx].e[d] = tri_edge[3 * tg + d];
      }
    }
  }
  __syncthreads();
  const int s = tile.src0 + threadIdx.x;
  if (s >= tk.nsrc) return;
  const int cg = tk.c0 + s;       // child id
  const int par = cg / 6, kk = cg % 6, pp = kk / 2;
  const int32_t cv = tri[3 * par + ((kk & 1) ? (pp + 1) % 3 : pp)];  // child's primal vertex
  const int32_t ce = tri_edge[3 * par + (pp + 2) % 3];                // edge of the child's midpoint
  const double* gs = bgeo + size_t(cg) * GEO_STRIDE;
  R rs[18], Ws[6], bv[9], sg_[3], cshi[3], cslo[3];
#pragma unroll
  for (int d = 0; d < 18; ++d) rs[d] = R(gs[GEO_RHO + d]);
#pragma unroll
  for (int d = 0; d < 6; ++d) Ws[d] = R(gs[GEO_W + d]);
#pragma unroll
  for (int d = 0; d < 9; ++d) bv[d] = R(gs[GEO_AV + d]);
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    sg_[d] = R(gs[GEO_SIG + d]);
    split_hl(gs[GEO_C + d], cshi[d], cslo[d]);
  }
  const int32_t be[3] = {btri_edge[3 * cg], btri_edge[3 * cg + 1], btri_edge[3 * cg + 2]};
  const R kr = R(tk.kr), ki = R(tk.ki);
#pragma unroll
  for (int k = 0; k < 6; ++k) Ws[k] *= R(INV4PI);  // 1/(4 pi) of grad G folded into the source weights

  for (int tt = 0; tt < tile_test<R>(); ++tt) {
    const int t = tile.test0 + tt;
    if (t >= tk.ntest) break;
    const TestRec<R>& X = T[tt];
    if (tk.t0 + t == par) continue;  // child of the test triangle: coplanar, Kbar = 0
    bool touch = false;
#pragma unroll
    for (int i = 0; i < 3; ++i) touch |= (X.v[i] == cv) | (X.e[i] == ce);
    if (touch) continue;  // FP64 extraction kernel
    const R dc0 = (X.chi[0] - cshi[0]) + (X.clo[0] - cslo[0]);
    const R dc1 = (X.chi[1] - cshi[1]) + (X.clo[1] - cslo[1]);
    const R dc2 = (X.chi[2] - cshi[2]) + (X.clo[2] - cslo[2]);
    R p1r = 0, p1i = 0, p2r[3] = {0, 0, 0}, p2i[3] = {0, 0, 0}, xr[3] = {0, 0, 0}, xi[3] = {0, 0, 0};
    R sr[3] = {0, 0, 0}, si[3] = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const R rqx = X.rho[3 * q], rqy = X.rho[3 * q + 1], rqz = X.rho[3 * q + 2];
      const R px = dc0 + rqx, py = dc1 + rqy, pz = dc2 + rqz;
      R ur[3] = {0, 0, 0}, ui[3] = {0, 0, 0}, vr[3] = {0, 0, 0}, vi[3] = {0, 0, 0};
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const R dx = px - rs[3 * k], dy = py - rs[3 * k + 1], dz = pz - rs[3 * k + 2];
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R ir = M<R>::rsqrt_(r2);
        const R Rr = r2 * ir;
        R sn, cn;
        M<R>::sincos_(kr * Rr, &sn, &cn);
        const R amp = (ki != R(0) ? M<R>::exp_(ki * Rr) : R(1)) * ir * ir * ir * Ws[k];
        // g1 = -(1 + j k R) exp(-j k R) / (4 pi R^3)
        const R er = amp * cn, ei = -amp * sn;
        const R ar = R(1) - ki * Rr, ai = kr * Rr;
        const R g1r = -(ar * er - ai * ei), g1i = -(ar * ei + ai * er);
        // D x rho'
        const R cx = dy * rs[3 * k + 2] - dz * rs[3 * k + 1];
        const R cy = dz * rs[3 * k] - dx * rs[3 * k + 2];
        const R cz = dx * rs[3 * k + 1] - dy * rs[3 * k];
        ur[0] += g1r * cx; ui[0] += g1i * cx;
        ur[1] += g1r * cy; ui[1] += g1i * cy;
        ur[2] += g1r * cz; ui[2] += g1i * cz;
        vr[0] += g1r * dx; vi[0] += g1i * dx;
        vr[1] += g1r * dy; vi[1] += g1i * dy;
        vr[2] += g1r * dz; vi[2] += g1i * dz;
      }
      const R w = X.W[q];
      p1r += w * (rqx * ur[0] + rqy * ur[1] + rqz * ur[2]);
      p1i += w * (rqx * ui[0] + rqy * ui[1] + rqz * ui[2]);
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        p2r[d] += w * ur[d];
        p2i[d] += w * ui[d];
        sr[d] += w * vr[d];
        si[d] += w * vi[d];
      }
      // rho_q x V
      xr[0] += w * (rqy * vr[2] - rqz * vr[1]); xi[0] += w * (rqy * vi[2] - rqz * vi[1]);
      xr[1] += w * (rqz * vr[0] - rqx * vr[2]); xi[1] += w * (rqz * vi[0] - rqx * vi[2]);
      xr[2] += w * (rqx * vr[1] - rqy * vr[0]); xi[2] += w * (rqx * vi[1] - rqy * vi[0]);
    }
    // local: sig_i sig'_j [P1 + a_i.P2 + b_j.X + b_j.(a_i x S)]
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R ax = X.av[3 * i], ay = X.av[3 * i + 1], az = X.av[3 * i + 2];
      const R baser = p1r + ax * p2r[0] + ay * p2r[1] + az * p2r[2];
      const R basei = p1i + ax * p2i[0] + ay * p2i[1] + az * p2i[2];
      // a_i x S
      const R csr0 = ay * sr[2] - az * sr[1], csr1 = az * sr[0] - ax * sr[2], csr2 = ax * sr[1] - ay * sr[0];
      const R csi0 = ay * si[2] - az * si[1], csi1 = az * si[0] - ax * si[2], csi2 = ax * si[1] - ay * si[0];
      const int64_t row = int64_t(X.e[i] - tk.e_row0) * tk.ld;
#pragma unroll
      for (int j = 0; j < 3; ++j) {
        const R bx = bv[3 * j], by = bv[3 * j + 1], bz = bv[3 * j + 2];
        R vr_ = baser + bx * (xr[0] + csr0) + by * (xr[1] + csr1) + bz * (xr[2] + csr2);
        R vi_ = basei + bx * (xi[0] + csi0) + by * (xi[1] + csi1) + bz * (xi[2] + csi2);
        const R sc = X.sig[i] * sg_[j];
        M<R>::add(tk.Kb, row + (be[j] - tk.b_col0), vr_ * sc, vi_ * sc);
      }
    }
  }
}

// ---------------------------------------------------------------- FP64 touching Kbar pairs
// Same lane layout as the L kernel: lane q < 6 takes outer point q.
template <class R>
__global__ void fill_K_touch(const KTask* __restrict__ tasks, const int32_t* __restrict__ obj_task,
                             const int32_t* __restrict__ tri_obj, const int32_t* __restrict__ pa,
                             const int32_t* __restrict__ pc, int npairs, const double* __restrict__ geo,
                             const double* __restrict__ bgeo, const double* __restrict__ xyz,
                             const int32_t* __restrict__ tri, const int32_t* __restrict__ tri_edge,
                             const int32_t* __restrict__ btri_edge) {
  const int64_t gt = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int p = int(gt >> 3), q = int(gt & 7);
  int task = -1, t = 0, cg = 0;
  if (p < npairs) {
    t = pa[p];
    cg = pc[p];
    task = obj_task[tri_obj[t]];
  }
  const bool act = task >= 0 && q < 6;
  KTask tk;
  if (task >= 0) tk = tasks[task];
  const double* gt_ = geo + size_t(t) * GEO_STRIDE;
  const double* gs = bgeo + size_t(cg) * GEO_STRIDE;
  double m[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = 0.0;
  if (act) {
    // child vertices rebuilt from the parent: (a, m_ab, g) (m_ab, b, g) (b, m_bc, g) (m_bc, c, g) (c, m_ca, g) (m_ca, a, g)
    const int par = cg / 6, kk = cg % 6;
    const double* a = xyz + 3 * tri[3 * par];
    const double* b = xyz + 3 * tri[3 * par + 1];
    const double* c = xyz + 3 * tri[3 * par + 2];
    double V[7][3];
    for (int d = 0; d < 3; ++d) {
      V[0][d] = a[d]; V[1][d] = b[d]; V[2][d] = c[d];
      V[3][d] = 0.5 * (a[d] + b[d]); V[4][d] = 0.5 * (b[d] + c[d]); V[5][d] = 0.5 * (c[d] + a[d]);
      V[6][d] = (a[d] + b[d] + c[d]) / 3.0;
    }
    const int cv[6][3] = {{0, 3, 6}, {3, 1, 6}, {1, 4, 6}, {4, 2, 6}, {2, 5, 6}, {5, 0, 6}};
    const cd k = {tk.kr, tk.ki};
    double r[3], rq[3];
    for (int d = 0; d < 3; ++d) {
      rq[d] = gt_[GEO_RHO + 3 * q + d];
      r[d] = gt_[GEO_C + d] + rq[d];
    }
    cd U[3] = {{0, 0}, {0, 0}, {0, 0}}, Vv[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int j = 0; j < 6; ++j) {
      const double* rs = gs + GEO_RHO + 3 * j;
      const double D[3] = {r[0] - gs[GEO_C] - rs[0], r[1] - gs[GEO_C + 1] - rs[1], r[2] - gs[GEO_C + 2] - rs[2]};
      cd g1 = grad_smooth(k, sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]));
      const double w = gs[GEO_W + j];
      g1.r *= w;
      g1.i *= w;
      const double cr[3] = {D[1] * rs[2] - D[2] * rs[1], D[2] * rs[0] - D[0] * rs[2], D[0] * rs[1] - D[1] * rs[0]};
      for (int d = 0; d < 3; ++d) {
        U[d].r += g1.r * cr[d];
        U[d].i += g1.i * cr[d];
        Vv[d].r += g1.r * D[d];
        Vv[d].i += g1.i * D[d];
      }
    }
    // static part: V_s = int grad 1/(4 pi R) dS', U_s = V_s x (r - c')
    Pot P;
    potentials(r, V[cv[kk][0]], V[cv[kk][1]], V[cv[kk][2]], P);
    double vs[3], rc[3];
    for (int d = 0; d < 3; ++d) {
      vs[d] = INV4PI * P.grad[d];
      rc[d] = r[d] - gs[GEO_C + d];
    }
    const double us[3] = {vs[1] * rc[2] - vs[2] * rc[1], vs[2] * rc[0] - vs[0] * rc[2], vs[0] * rc[1] - vs[1] * rc[0]};
    for (int d = 0; d < 3; ++d) {
      U[d].r += us[d];
      Vv[d].r += vs[d];
    }
    const double w = gt_[GEO_W + q];
    for (int d = 0; d < 3; ++d) {
      m[0] += w * rq[d] * U[d].r;            // P1
      m[1] += w * rq[d] * U[d].i;
      m[2 + 2 * d] = w * U[d].r;             // P2
      m[3 + 2 * d] = w * U[d].i;
      m[14 + 2 * d] = w * Vv[d].r;           // S
      m[15 + 2 * d] = w * Vv[d].i;
    }
    // X = rho x V
    m[8] = w * (rq[1] * Vv[2].r - rq[2] * Vv[1].r);  m[9] = w * (rq[1] * Vv[2].i - rq[2] * Vv[1].i);
    m[10] = w * (rq[2] * Vv[0].r - rq[0] * Vv[2].r); m[11] = w * (rq[2] * Vv[0].i - rq[0] * Vv[2].i);
    m[12] = w * (rq[0] * Vv[1].r - rq[1] * Vv[0].r); m[13] = w * (rq[0] * Vv[1].i - rq[1] * Vv[0].i);
  }
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = grp_sum8(m[i]);
  if (task < 0 || q != 0) return;
  const cd P1 = {m[0], m[1]};
  cd P2[3], X[3], S[3];
  for (int d = 0; d < 3; ++d) {
    P2[d] = {m[2 + 2 * d], m[3 + 2 * d]};
    X[d] = {m[8 + 2 * d], m[9 + 2 * d]};
    S[d] = {m[14 + 2 * d], m[15 + 2 * d]};
  }
  for (int i = 0; i < 3; ++i) {
    const double* av = gt_ + GEO_AV + 3 * i;
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
      const double sc = gt_[GEO_SIG + i] * gs[GEO_SIG + j];
      add_d<R>(tk.Kb, int64_t(tri_edge[3 * t + i] - tk.e_row0) * tk.ld + (btri_edge[3 * cg + j] - tk.b_col0), v.r * sc,
               v.i * sc);
    }
  }
}

// ---------------------------------------------------------------- host launchers
// Task of each object's touching pairs: the first task whose test-triangle and
// source ranges both hold the object (tasks cover whole objects), or -1 (an
// object whose own block no task fills).
static int32_t src_begin(const LTask& t) { return t.s0; }
static int32_t src_end(const LTask& t) { return t.s0 + t.nsrc; }
static int32_t src_begin(const KTask& t) { return t.c0 / 6; }
static int32_t src_end(const KTask& t) { return (t.c0 + t.nsrc) / 6; }
template <class T>
static std::vector<int32_t> object_tasks(const HostMesh& h, const std::vector<T>& tasks) {
  std::vector<int32_t> ot(size_t(h.nobj), -1);
  for (int64_t o = 0; o < h.nobj; ++o)
    for (size_t i = 0; i < tasks.size(); ++i) {
      const int32_t b = h.tri_begin[o];
      if (b >= tasks[i].t0 && b < tasks[i].t0 + tasks[i].ntest && b >= src_begin(tasks[i]) && b < src_end(tasks[i])) {
        ot[size_t(o)] = int32_t(i);
        break;
      }
    }
  return ot;
}

// Tasks with a source split for a good conductor go to the split kernels whole
// (their touching pairs included); the others to the bulk and touching kernels.
template <class T>
static std::vector<int32_t> unsplit_object_tasks(const HostMesh& h, const std::vector<T>& tasks, const std::vector<char>& split) {
  std::vector<int32_t> ot = object_tasks(h, tasks);
  for (auto& o : ot)
    if (o >= 0 && split[size_t(o)]) o = -1;
  return ot;
}

template <class R>
void fill_L(const sldm_mesh* m, const std::vector<LTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  std::vector<SplitRules> rules(tasks.size());
  std::vector<char> split(tasks.size(), 0);
  for (size_t i = 0; i < tasks.size(); ++i) {
    rules[i] = split_rules_L(m->h, tasks[i]);
    split[i] = rules[i].split;
  }
  std::vector<TileRef> tiles;
  for (size_t i = 0; i < tasks.size(); ++i) {
    if (split[i]) continue;
    for (int t0 = 0; t0 < tasks[i].ntest; t0 += tile_test<R>())
      for (int s0 = 0; s0 < tasks[i].nsrc; s0 += TILE_SRC) tiles.push_back({int32_t(i), t0, s0, 0});
  }
  DBuf<LTask> dt;
  DBuf<TileRef> dtl;
  dt.upload(tasks, s);
  dtl.upload(tiles, s);
  const DevMesh& d = m->d;
  const std::vector<int32_t> ot = unsplit_object_tasks(m->h, tasks, split);
  if (timers_on()) {  // evaluations of the bulk kernel: 36 per non-touching pair of the unsplit tasks
    double pairs = 0;
    for (size_t i = 0; i < tasks.size(); ++i)
      if (!split[i]) pairs += double(tasks[i].ntest) * tasks[i].nsrc;
    for (size_t k = 0; k < m->h.touchL_a.size(); ++k)
      if (ot[size_t(m->h.obj[m->h.touchL_a[k]])] >= 0) pairs -= 1;
    timer_units("fill_L_bulk", 36.0 * pairs);
  }
  for (size_t off = 0; off < tiles.size(); off += 1u << 30) {
    unsigned nb = unsigned(std::min<size_t>(tiles.size() - off, 1u << 30));
    ScopedTimer tm("fill_L_bulk", s);
    fill_L_bulk<R><<<nb, TILE_SRC, 0, s>>>(dt.p, dtl.p + off, d.geo.p, d.tri.p, d.tri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  const int np = int(m->h.touchL_a.size());
  DBuf<int32_t> dot;
  dot.upload(ot, s);
  if (np > 0) {
    ScopedTimer tm("fill_L_touch", s);
    fill_L_touch<R><<<unsigned((int64_t(np) * 8 + 255) / 256), 256, 0, s>>>(dt.p, dot.p, d.obj.p, d.touchL_a.p, d.touchL_b.p, np,
                                                                            d.geo.p, d.xyz.p, d.tri.p, d.tri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  for (size_t i = 0; i < tasks.size(); ++i)
    if (split[i]) fill_L_split_task<R>(m, tasks[i], rules[i], s);
  SLDM_CUDA(cudaStreamSynchronize(s));  // task/tile buffers are released on return
}

template <class R>
void fill_K(const sldm_mesh* m, const std::vector<KTask>& tasks, cudaStream_t s) {
  if (tasks.empty()) return;
  std::vector<SplitRules> rules(tasks.size());
  std::vector<char> split(tasks.size(), 0);
  for (size_t i = 0; i < tasks.size(); ++i) {
    rules[i] = split_rules_K(m->h, tasks[i]);
    split[i] = rules[i].split;
  }
  std::vector<TileRef> tiles;
  for (size_t i = 0; i < tasks.size(); ++i) {
    if (split[i]) continue;
    for (int t0 = 0; t0 < tasks[i].ntest; t0 += tile_test<R>())
      for (int s0 = 0; s0 < tasks[i].nsrc; s0 += TILE_SRC) tiles.push_back({int32_t(i), t0, s0, 0});
  }
  DBuf<KTask> dt;
  DBuf<TileRef> dtl;
  dt.upload(tasks, s);
  dtl.upload(tiles, s);
  const DevMesh& d = m->d;
  if (timers_on()) {  // evaluations of the bulk kernel: 36 per pair that is neither a child of its test triangle nor touching
    const std::vector<int32_t> ot = unsplit_object_tasks(m->h, tasks, split);
    double pairs = 0;
    for (size_t i = 0; i < tasks.size(); ++i)
      if (!split[i]) pairs += double(tasks[i].ntest) * tasks[i].nsrc;
    for (int64_t o = 0; o < m->h.nobj; ++o)
      if (ot[size_t(o)] >= 0) pairs -= 6.0 * (m->h.tri_begin[o + 1] - m->h.tri_begin[o]);
    for (size_t k = 0; k < m->h.touchK_a.size(); ++k)
      if (ot[size_t(m->h.obj[m->h.touchK_a[k]])] >= 0) pairs -= 1;
    timer_units("fill_K_bulk", 36.0 * pairs);
  }
  if (!tiles.empty()) {
    ScopedTimer tm("fill_K_bulk", s);
    fill_K_bulk<R><<<unsigned(tiles.size()), TILE_SRC, 0, s>>>(dt.p, dtl.p, d.geo.p, d.bgeo.p, d.tri.p, d.tri_edge.p,
                                                             d.btri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  const int np = int(m->h.touchK_a.size());
  DBuf<int32_t> dot;
  dot.upload(unsplit_object_tasks(m->h, tasks, split), s);
  if (np > 0) {
    ScopedTimer tm("fill_K_touch", s);
    fill_K_touch<R><<<unsigned((int64_t(np) * 8 + 255) / 256), 256, 0, s>>>(dt.p, dot.p, d.obj.p, d.touchK_a.p, d.touchK_c.p, np,
                                                                            d.geo.p, d.bgeo.p, d.xyz.p, d.tri.p, d.tri_edge.p,
                                                                            d.btri_edge.p), ::sldm::count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
  for (size_t i = 0; i < tasks.size(); ++i)
    if (split[i]) fill_K_split_task<R>(m, tasks[i], rules[i], s);
  SLDM_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- BC contraction
// K[m][n] = sum_q Kb[m][row_q - b0] * val_q over the CSC column n of C.
template <class R>
__global__ void contract_bc_kernel(int ne_o, int e0, int b0, const int32_t* __restrict__ ptr, const int32_t* __restrict__ row,
                                   const double* __restrict__ val, const void* __restrict__ Kb_, int64_t ldKb, void* K_,
                                   int64_t ldK) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  int m = blockIdx.y;
  if (n >= ne_o) return;
  typedef typename std::conditional<sizeof(R) == 4, float2, double2>::type C2;
  const C2* Kb = reinterpret_cast<const C2*>(Kb_) + int64_t(m) * ldKb;
  double sr = 0, si = 0;
  for (int q = ptr[e0 + n]; q < ptr[e0 + n + 1]; ++q) {
    C2 v = Kb[row[q] - b0];
    sr += double(v.x) * val[q];
    si += double(v.y) * val[q];
  }
  C2* K = reinterpret_cast<C2*>(K_) + int64_t(m) * ldK;
  K[n].x = decltype(K[n].x)(sr);
  K[n].y = decltype(K[n].y)(si);
}

template <class R>
void contract_bc(const sldm_mesh* m, int obj, const void* Kb, int64_t ldKb, void* K, int64_t ldK, cudaStream_t s) {
  const HostMesh& h = m->h;
  int e0 = h.edge_begin[obj], ne_o = h.edge_begin[obj + 1] - e0;
  int b0 = h.bedge_begin[obj];
  dim3 grid((ne_o + 127) / 128, ne_o);
  contract_bc_kernel<R><<<grid, 128, 0, s>>>(ne_o, e0, b0, m->d.bc_ptr.p, m->d.bc_row.p, m->d.bc_val.p, Kb, ldKb, K, ldK), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- Gram I_x
// value of nonzero z: sum over its contributions of coef * int_child (n_T x f_i) . g_j (6-point, exact)
__global__ void gram_kernel(int nnz, const int32_t* __restrict__ cptr, const int32_t* __restrict__ ctri,
                            const int32_t* __restrict__ cchild, const int32_t* __restrict__ ci,
                            const int32_t* __restrict__ cj, const double* __restrict__ ccoef,
                            const double* __restrict__ geo, const double* __restrict__ bgeo, double* vals) {
  int z = blockIdx.x * blockDim.x + threadIdx.x;
  if (z >= nnz) return;
  double acc = 0;
  for (int q = cptr[z]; q < cptr[z + 1]; ++q) {
    const double* gt = geo + size_t(ctri[q]) * GEO_STRIDE;
    const double* gc = bgeo + size_t(cchild[q]) * GEO_STRIDE;
    int i = ci[q], j = cj[q];
    const double* n = gt + GEO_N;
    double sum = 0;
    for (int p = 0; p < 6; ++p) {
      double r[3], f[3], g[3];
      for (int d = 0; d < 3; ++d) {
        r[d] = gc[GEO_C + d] + gc[GEO_RHO + 3 * p + d];
        f[d] = gt[GEO_SIG + i] * (r[d] - gt[GEO_C + d] + gt[GEO_AV + 3 * i + d]);
        g[d] = gc[GEO_SIG + j] * (gc[GEO_RHO + 3 * p + d] + gc[GEO_AV + 3 * j + d]);
      }
      double nf[3] = {n[1] * f[2] - n[2] * f[1], n[2] * f[0] - n[0] * f[2], n[0] * f[1] - n[1] * f[0]};
      sum += gc[GEO_W + p] * (nf[0] * g[0] + nf[1] * g[1] + nf[2] * g[2]);
    }
    acc += ccoef[q] * sum;
  }
  vals[z] = acc;
}

void gram_ix(const sldm_mesh* m, double* vals, cudaStream_t s) {
  int nnz = int(m->h.ix_col.size());
  const DevMesh& d = m->d;
  gram_kernel<<<(nnz + 127) / 128, 128, 0, s>>>(nnz, d.ixc_ptr.p, d.ixc_tri.p, d.ixc_child.p, d.ixc_i.p, d.ixc_j.p,
                                                d.ixc_coef.p, d.geo.p, d.bgeo.p, vals), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- plane-wave right-hand side
constexpr double ETA0 = 4e-7 * PI * 299792458.0;

__global__ void rhs_kernel(int ne, int nrhs, double k0, const double* __restrict__ kp, const int32_t* __restrict__ tplus,
                           const int32_t* __restrict__ tminus, const int32_t* __restrict__ tri_edge,
                           const double* __restrict__ geo, double2* b, int64_t ld) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (m >= ne) return;
  const double* kh = kp + 6 * r;
  const double* pol = kh + 3;
  double acc_r = 0, acc_i = 0;
  for (int side = 0; side < 2; ++side) {
    int t = side == 0 ? tplus[m] : tminus[m];
    const double* g = geo + size_t(t) * GEO_STRIDE;
    int i = tri_edge[3 * t] == m ? 0 : (tri_edge[3 * t + 1] == m ? 1 : 2);
    for (int q = 0; q < 6; ++q) {
      double fp = 0, ph = 0;
      for (int d = 0; d < 3; ++d) {
        double rl = g[GEO_RHO + 3 * q + d];
        fp += g[GEO_SIG + i] * (rl + g[GEO_AV + 3 * i + d]) * pol[d];
        ph += kh[d] * (g[GEO_C + d] + rl);
      }
      double sn, cn;
      sincos(k0 * ph, &sn, &cn);
      double w = g[GEO_W + q] * fp / ETA0;
      acc_r += w * cn;
      acc_i -= w * sn;
    }
  }
  b[int64_t(r) * ld + m] = make_double2(acc_r, acc_i);
}

// Plane wave through a stack, in the objects' layer (record layout PW_*):
// E = e^{-j kt.r} [phi V_TE + rho V_TM + z (|kt| / k_z)(a_TM e^+ - c_TM e^-)],
// V = a e^+ + c e^-, e^{+-} = e^{+-j k_z (z - zref)}, phi = z x rho.
__device__ void stack_wave(const double* __restrict__ P, const double x[3], double er[3], double ei[3]) {
  const double ktx = P[PW_KT], kty = P[PW_KT + 1], rx = P[PW_RHO], ry = P[PW_RHO + 1];
  const double px = -ry, py = rx;
  const double kr = P[PW_KZ], ki = P[PW_KZ + 1];
  const double kn = kr * kr + ki * ki;
  const double qr = P[PW_KRHO] * kr / kn, qi = -P[PW_KRHO] * ki / kn;  // |kt| / k_z
  const double dz = x[2] - P[PW_ZREF];
  // e^{+j k_z dz} = e^{-ki dz} (cos(kr dz) + j sin(kr dz)),  e^{-j k_z dz} = e^{ki dz} (cos - j sin)
  double sn, cn;
  sincos(kr * dz, &sn, &cn);
  const double ep = exp(-ki * dz), em = exp(ki * dz);
  const double ur = ep * cn, ui = ep * sn, vr = em * cn, vi = -em * sn;
  const double ater = P[PW_A], atei = P[PW_A + 1], cter = P[PW_A + 2], ctei = P[PW_A + 3];
  const double atmr = P[PW_A + 4], atmi = P[PW_A + 5], ctmr = P[PW_A + 6], ctmi = P[PW_A + 7];
  const double vte_r = ater * ur - atei * ui + cter * vr - ctei * vi;
  const double vte_i = ater * ui + atei * ur + cter * vi + ctei * vr;
  const double vtm_r = atmr * ur - atmi * ui + ctmr * vr - ctmi * vi;
  const double vtm_i = atmr * ui + atmi * ur + ctmr * vi + ctmi * vr;
  const double dr = atmr * ur - atmi * ui - (ctmr * vr - ctmi * vi);
  const double di = atmr * ui + atmi * ur - (ctmr * vi + ctmi * vr);
  const double ez_r = qr * dr - qi * di, ez_i = qr * di + qi * dr;
  double sl, cl;  // e^{-j kt.r}
  sincos(ktx * x[0] + kty * x[1], &sl, &cl);
  const double fr[3] = {px * vte_r + rx * vtm_r, py * vte_r + ry * vtm_r, ez_r};
  const double fi[3] = {px * vte_i + rx * vtm_i, py * vte_i + ry * vtm_i, ez_i};
  for (int d = 0; d < 3; ++d) {
    er[d] = fr[d] * cl + fi[d] * sl;
    ei[d] = fi[d] * cl - fr[d] * sl;
  }
}

__global__ void rhs_layered_kernel(int ne, const double* __restrict__ rec, const int32_t* __restrict__ tplus,
                                   const int32_t* __restrict__ tminus, const int32_t* __restrict__ tri_edge,
                                   const double* __restrict__ geo, double2* b, int64_t ld) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (m >= ne) return;
  const double* P = rec + size_t(r) * PW_REC;
  double acc_r = 0, acc_i = 0;
  for (int side = 0; side < 2; ++side) {
    int t = side == 0 ? tplus[m] : tminus[m];
    const double* g = geo + size_t(t) * GEO_STRIDE;
    int i = tri_edge[3 * t] == m ? 0 : (tri_edge[3 * t + 1] == m ? 1 : 2);
    for (int q = 0; q < 6; ++q) {
      double f[3], x[3], er[3], ei[3];
      for (int d = 0; d < 3; ++d) {
        f[d] = g[GEO_SIG + i] * (g[GEO_RHO + 3 * q + d] + g[GEO_AV + 3 * i + d]);
        x[d] = g[GEO_C + d] + g[GEO_RHO + 3 * q + d];
      }
      stack_wave(P, x, er, ei);
      const double w = g[GEO_W + q] / ETA0;
      acc_r += w * (f[0] * er[0] + f[1] * er[1] + f[2] * er[2]);
      acc_i += w * (f[0] * ei[0] + f[1] * ei[1] + f[2] * ei[2]);
    }
  }
  b[int64_t(r) * ld + m] = make_double2(acc_r, acc_i);
}

void rhs_planewave_layered(const sldm_mesh* m, const double* rec, int nrhs, double2* b, int64_t ld, cudaStream_t s) {
  int ne = int(m->h.ne);
  dim3 grid((ne + 127) / 128, nrhs);
  rhs_layered_kernel<<<grid, 128, 0, s>>>(ne, rec, m->d.tplus.p, m->d.tminus.p, m->d.tri_edge.p, m->d.geo.p, b, ld),
      ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

void rhs_planewave(const sldm_mesh* m, double k0, const double* kp, int nrhs, double2* b, int64_t ld, cudaStream_t s) {
  int ne = int(m->h.ne);
  dim3 grid((ne + 127) / 128, nrhs);
  rhs_kernel<<<grid, 128, 0, s>>>(ne, nrhs, k0, kp, m->d.tplus.p, m->d.tminus.p, m->d.tri_edge.p, m->d.geo.p, b, ld), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- far field / RCS
// Right-hand sides per CTA of the far-field kernels: the phase factors (or the
// stack's waves) at a quadrature point are computed once for all of them.
constexpr int FF_NR = 8;
constexpr int FF_THREADS = 128;

// Sum of NV per-thread values over the CTA (warp shuffles, then one value per
// warp in shared memory); the totals land in out[] of thread 0.
template <int NV>
__device__ __forceinline__ void ff_reduce(double* v, double (*sh)[NV], double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < NV; ++c) {
    double x = v[c];
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) sh[warp][c] = x;
  }
  __syncthreads();
  if (threadIdx.x == 0)
    for (int c = 0; c < NV; ++c) {
      double x = 0;
      for (int w = 0; w < FF_THREADS / 32; ++w) x += sh[w][c];
      out[c] = x;
    }
}

// F_r = sum_m jd_r,m int f_m exp(+j k0 rhat . r); sigma = eta0^2 |(I - rr) F_r|^2 / (4 pi)
// CTA (a, g): angle a, right-hand sides [g FF_NR, g FF_NR + cnt); jd column r at jd + r ldj
__global__ void __launch_bounds__(FF_THREADS) farfield_kernel(int nt, double k0, const double2* __restrict__ jd, int64_t ldj,
                                                              int nr, const int32_t* __restrict__ tri_edge,
                                                              const double* __restrict__ geo, const double* __restrict__ ang,
                                                              int n, double* rcs) {
  const int a = blockIdx.x, r0 = blockIdx.y * FF_NR;
  const int cnt = min(FF_NR, nr - r0);
  const double th = ang[2 * a], ph = ang[2 * a + 1];
  const double rh[3] = {sin(th) * cos(ph), sin(th) * sin(ph), cos(th)};
  double F[6 * FF_NR];
#pragma unroll
  for (int c = 0; c < 6 * FF_NR; ++c) F[c] = 0;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double* g = geo + size_t(t) * GEO_STRIDE;
    for (int q = 0; q < 6; ++q) {
      double pr = 0;
      for (int d = 0; d < 3; ++d) pr += rh[d] * (g[GEO_C + d] + g[GEO_RHO + 3 * q + d]);
      double sn, cn;
      sincos(k0 * pr, &sn, &cn);
      for (int i = 0; i < 3; ++i) {
        const int e = tri_edge[3 * t + i];
        const double wr = g[GEO_W + q] * g[GEO_SIG + i];
        double f[3];
        for (int d = 0; d < 3; ++d) f[d] = g[GEO_RHO + 3 * q + d] + g[GEO_AV + 3 * i + d];
#pragma unroll
        for (int r = 0; r < FF_NR; ++r) {
          if (r >= cnt) break;
          const double2 c = jd[int64_t(r0 + r) * ldj + e];
          // c exp(+j k0 rhat.r)
          const double er = (c.x * cn - c.y * sn) * wr, ei = (c.x * sn + c.y * cn) * wr;
          for (int d = 0; d < 3; ++d) {
            F[6 * r + 2 * d] += er * f[d];
            F[6 * r + 2 * d + 1] += ei * f[d];
          }
        }
      }
    }
  }
  __shared__ double sh[FF_THREADS / 32][6 * FF_NR];
  __shared__ double tot[6 * FF_NR];
  ff_reduce<6 * FF_NR>(F, sh, tot);
  if (threadIdx.x != 0) return;
  for (int r = 0; r < cnt; ++r) {
    const double* fr = tot + 6 * r;
    const double dr = rh[0] * fr[0] + rh[1] * fr[2] + rh[2] * fr[4];
    const double di = rh[0] * fr[1] + rh[1] * fr[3] + rh[2] * fr[5];
    double s2 = 0;
    for (int d = 0; d < 3; ++d) {
      const double pr_ = fr[2 * d] - rh[d] * dr, pi_ = fr[2 * d + 1] - rh[d] * di;
      s2 += pr_ * pr_ + pi_ * pi_;
    }
    rcs[int64_t(r0 + r) * n + a] = ETA0 * ETA0 * s2 / (4 * PI);
  }
}

void farfield(const sldm_mesh* m, double k0, const double2* jd, int64_t ldj, int nr, const double* ang, int n, double* rcs,
              cudaStream_t s) {
  farfield_kernel<<<dim3(n, (nr + FF_NR - 1) / FF_NR), FF_THREADS, 0, s>>>(int(m->h.nt), k0, jd, ldj, nr, m->d.tri_edge.p,
                                                                           m->d.geo.p, ang, n, rcs),
      ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// Far field above a stack: for angle a, the reaction of the currents with the
// stack's plane waves arriving from the observation direction, theta- and
// phi-polarised (records rec[2a], rec[2a + 1]);  sigma = eta0^2 (|F_t|^2 + |F_p|^2) / (4 pi)
__global__ void __launch_bounds__(FF_THREADS) farfield_layered_kernel(int nt, const double2* __restrict__ jd, int64_t ldj,
                                                                      int nr, const int32_t* __restrict__ tri_edge,
                                                                      const double* __restrict__ geo,
                                                                      const double* __restrict__ rec, int n, double* rcs) {
  const int a = blockIdx.x, r0 = blockIdx.y * FF_NR;
  const int cnt = min(FF_NR, nr - r0);
  const double* P0 = rec + size_t(2 * a) * PW_REC;
  const double* P1 = P0 + PW_REC;
  double F[4 * FF_NR];
#pragma unroll
  for (int c = 0; c < 4 * FF_NR; ++c) F[c] = 0;
  for (int t = threadIdx.x; t < nt; t += blockDim.x) {
    const double* g = geo + size_t(t) * GEO_STRIDE;
    for (int q = 0; q < 6; ++q) {
      double x[3];
      for (int d = 0; d < 3; ++d) x[d] = g[GEO_C + d] + g[GEO_RHO + 3 * q + d];
      double e0r[3], e0i[3], e1r[3], e1i[3];
      stack_wave(P0, x, e0r, e0i);
      stack_wave(P1, x, e1r, e1i);
      for (int i = 0; i < 3; ++i) {
        const int e = tri_edge[3 * t + i];
        const double w = g[GEO_W + q] * g[GEO_SIG + i];
        double p0r = 0, p0i = 0, p1r = 0, p1i = 0;  // f_i . E_p
        for (int d = 0; d < 3; ++d) {
          const double f = g[GEO_RHO + 3 * q + d] + g[GEO_AV + 3 * i + d];
          p0r += f * e0r[d];
          p0i += f * e0i[d];
          p1r += f * e1r[d];
          p1i += f * e1i[d];
        }
#pragma unroll
        for (int r = 0; r < FF_NR; ++r) {
          if (r >= cnt) break;
          const double2 c = jd[int64_t(r0 + r) * ldj + e];
          F[4 * r] += w * (c.x * p0r - c.y * p0i);
          F[4 * r + 1] += w * (c.x * p0i + c.y * p0r);
          F[4 * r + 2] += w * (c.x * p1r - c.y * p1i);
          F[4 * r + 3] += w * (c.x * p1i + c.y * p1r);
        }
      }
    }
  }
  __shared__ double sh[FF_THREADS / 32][4 * FF_NR];
  __shared__ double tot[4 * FF_NR];
  ff_reduce<4 * FF_NR>(F, sh, tot);
  if (threadIdx.x != 0) return;
  for (int r = 0; r < cnt; ++r) {
    const double* fr = tot + 4 * r;
    rcs[int64_t(r0 + r) * n + a] = ETA0 * ETA0 * (fr[0] * fr[0] + fr[1] * fr[1] + fr[2] * fr[2] + fr[3] * fr[3]) / (4 * PI);
  }
}

void farfield_layered(const sldm_mesh* m, const double2* jd, int64_t ldj, int nr, const double* rec, int n, double* rcs,
                      cudaStream_t s) {
  farfield_layered_kernel<<<dim3(n, (nr + FF_NR - 1) / FF_NR), FF_THREADS, 0, s>>>(int(m->h.nt), jd, ldj, nr, m->d.tri_edge.p,
                                                                                   m->d.geo.p, rec, n, rcs),
      ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

template void fill_L<float>(const sldm_mesh*, const std::vector<LTask>&, cudaStream_t);
template void fill_L<double>(const sldm_mesh*, const std::vector<LTask>&, cudaStream_t);
template void fill_K<float>(const sldm_mesh*, const std::vector<KTask>&, cudaStream_t);
template void fill_K<double>(const sldm_mesh*, const std::vector<KTask>&, cudaStream_t);
template void contract_bc<float>(const sldm_mesh*, int, const void*, int64_t, void*, int64_t, cudaStream_t);
template void contract_bc<double>(const sldm_mesh*, int, const void*, int64_t, void*, int64_t, cudaStream_t);

}  // namespace sldm

namespace sldm {

// ---------------------------------------------------------------- FP64 touching Kbar pairs, one task by value
// One thread per pair (used by the allocation-free entry point).
__global__ void fill_K_touch_one(KTask tk, const int32_t* __restrict__ pa, const int32_t* __restrict__ pc, int npairs,
                             const double* __restrict__ geo, const double* __restrict__ bgeo,
                             const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                             const int32_t* __restrict__ tri_edge, const int32_t* __restrict__ btri_edge) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npairs) return;
  const int t = pa[p], cg = pc[p];
  if (t < tk.t0 || t >= tk.t0 + tk.ntest || cg < tk.c0 || cg >= tk.c0 + tk.nsrc) return;
  const double* gt = geo + size_t(t) * GEO_STRIDE;
  const double* gs = bgeo + size_t(cg) * GEO_STRIDE;
  // child vertices: rebuild from the parent (a, m_ab, g) ... pattern
  const int par = cg / 6, kk = cg % 6;
  const double* a = xyz + 3 * tri[3 * par];
  const double* b = xyz + 3 * tri[3 * par + 1];
  const double* c = xyz + 3 * tri[3 * par + 2];
  double V[7][3];  // a, b, c, m_ab, m_bc, m_ca, g
  for (int d = 0; d < 3; ++d) {
    V[0][d] = a[d]; V[1][d] = b[d]; V[2][d] = c[d];
    V[3][d] = 0.5 * (a[d] + b[d]); V[4][d] = 0.5 * (b[d] + c[d]); V[5][d] = 0.5 * (c[d] + a[d]);
    V[6][d] = (a[d] + b[d] + c[d]) / 3.0;
  }
  const int cv[6][3] = {{0, 3, 6}, {3, 1, 6}, {1, 4, 6}, {4, 2, 6}, {2, 5, 6}, {5, 0, 6}};
  const double* p1 = V[cv[kk][0]];
  const double* p2 = V[cv[kk][1]];
  const double* p3 = V[cv[kk][2]];
  const cd k = {tk.kr, tk.ki};
  cd P1 = {0, 0}, P2[3] = {{0, 0}, {0, 0}, {0, 0}}, X[3] = {{0, 0}, {0, 0}, {0, 0}}, S[3] = {{0, 0}, {0, 0}, {0, 0}};
  for (int q = 0; q < 6; ++q) {
    double r[3], rq[3];
    for (int d = 0; d < 3; ++d) {
      rq[d] = gt[GEO_RHO + 3 * q + d];
      r[d] = gt[GEO_C + d] + rq[d];
    }
    cd U[3] = {{0, 0}, {0, 0}, {0, 0}}, Vv[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int j = 0; j < 6; ++j) {
      const double* rs = gs + GEO_RHO + 3 * j;
      double D[3] = {r[0] - gs[GEO_C] - rs[0], r[1] - gs[GEO_C + 1] - rs[1], r[2] - gs[GEO_C + 2] - rs[2]};
      double Rr = sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      cd g1 = grad_smooth(k, Rr);
      double w = gs[GEO_W + j];
      g1.r *= w;
      g1.i *= w;
      double cr[3] = {D[1] * rs[2] - D[2] * rs[1], D[2] * rs[0] - D[0] * rs[2], D[0] * rs[1] - D[1] * rs[0]};
      for (int d = 0; d < 3; ++d) {
        U[d].r += g1.r * cr[d];
        U[d].i += g1.i * cr[d];
        Vv[d].r += g1.r * D[d];
        Vv[d].i += g1.i * D[d];
      }
    }
    // static part: V_s = int grad 1/(4 pi R) dS', U_s = V_s x (r - c')
    Pot P;
    potentials(r, p1, p2, p3, P);
    double vs[3], rc[3];
    for (int d = 0; d < 3; ++d) {
      vs[d] = INV4PI * P.grad[d];
      rc[d] = r[d] - gs[GEO_C + d];
    }
    double us[3] = {vs[1] * rc[2] - vs[2] * rc[1], vs[2] * rc[0] - vs[0] * rc[2], vs[0] * rc[1] - vs[1] * rc[0]};
    for (int d = 0; d < 3; ++d) {
      U[d].r += us[d];
      Vv[d].r += vs[d];
    }
    double w = gt[GEO_W + q];
    for (int d = 0; d < 3; ++d) {
      P1.r += w * rq[d] * U[d].r;
      P1.i += w * rq[d] * U[d].i;
      P2[d].r += w * U[d].r;
      P2[d].i += w * U[d].i;
      S[d].r += w * Vv[d].r;
      S[d].i += w * Vv[d].i;
    }
    X[0].r += w * (rq[1] * Vv[2].r - rq[2] * Vv[1].r); X[0].i += w * (rq[1] * Vv[2].i - rq[2] * Vv[1].i);
    X[1].r += w * (rq[2] * Vv[0].r - rq[0] * Vv[2].r); X[1].i += w * (rq[2] * Vv[0].i - rq[0] * Vv[2].i);
    X[2].r += w * (rq[0] * Vv[1].r - rq[1] * Vv[0].r); X[2].i += w * (rq[0] * Vv[1].i - rq[1] * Vv[0].i);
  }
  for (int i = 0; i < 3; ++i) {
    const double* av = gt + GEO_AV + 3 * i;
    cd base = P1;
    for (int d = 0; d < 3; ++d) {
      base.r += av[d] * P2[d].r;
      base.i += av[d] * P2[d].i;
    }
    cd axs[3] = {{av[1] * S[2].r - av[2] * S[1].r, av[1] * S[2].i - av[2] * S[1].i},
                 {av[2] * S[0].r - av[0] * S[2].r, av[2] * S[0].i - av[0] * S[2].i},
                 {av[0] * S[1].r - av[1] * S[0].r, av[0] * S[1].i - av[1] * S[0].i}};
    for (int j = 0; j < 3; ++j) {
      const double* bv = gs + GEO_AV + 3 * j;
      cd v = base;
      for (int d = 0; d < 3; ++d) {
        v.r += bv[d] * (X[d].r + axs[d].r);
        v.i += bv[d] * (X[d].i + axs[d].i);
      }
      double sc = gt[GEO_SIG + i] * gs[GEO_SIG + j];
      add_d<double>(tk.Kb, int64_t(tri_edge[3 * t + i] - tk.e_row0) * tk.ld + (btri_edge[3 * cg + j] - tk.b_col0), v.r * sc,
               v.i * sc);
    }
  }
}

}  // namespace sldm

// ---------------------------------------------------------------- allocation-free Kbar
// sldm_kbar_noalloc: the barycentric Kbar fill of one object and its contraction
// with the BC coefficients, with every temporary (task record, tile list and the
// barycentric scratch block) in one file-scope device array instead of memory
// obtained from cudaMalloc.
namespace sldm {

constexpr size_t NOALLOC_BYTES = size_t(24) << 20;         // 24 MiB held on each GPU that loads this module
constexpr size_t NOALLOC_TASK_OFF = 0;                       // one KTask
constexpr size_t NOALLOC_TILE_OFF = 256;                     // TileRef[NOALLOC_MAX_TILES]
constexpr size_t NOALLOC_MAX_TILES = 4096;
constexpr size_t NOALLOC_KB_OFF = NOALLOC_TILE_OFF + NOALLOC_MAX_TILES * sizeof(TileRef);  // complex128 block
constexpr size_t NOALLOC_MAX_KB = (NOALLOC_BYTES - NOALLOC_KB_OFF) / sizeof(double2);

static_assert(sizeof(KTask) <= NOALLOC_TILE_OFF - NOALLOC_TASK_OFF, "task record overlaps the tile list");
static_assert(NOALLOC_TILE_OFF % alignof(TileRef) == 0, "tile list misaligned");
static_assert(NOALLOC_KB_OFF % alignof(double2) == 0 && NOALLOC_KB_OFF % 16 == 0, "scratch block misaligned");
static_assert(NOALLOC_KB_OFF < NOALLOC_BYTES, "no room for the scratch block");

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

// Device address of g_noalloc_scratch per device, resolved once with that device current.
static std::mutex g_noalloc_mu;
static void* g_noalloc_ptr[64] = {nullptr};

static void* noalloc_scratch(int dev) {
  SLDM_REQUIRE(dev >= 0 && dev < 64, SLDM_EINVAL, "kbar_noalloc: device index out of range");
  std::lock_guard<std::mutex> l(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    SLDM_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_ptr[dev] = p;
  }
  return g_noalloc_ptr[dev];
}

// Writes the task record and the tile list of one object into the scratch.
__global__ void noalloc_setup_kernel(KTask task, int ntile_t, int ntile_s, KTask* dtask, TileRef* dtiles) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *dtask = task;
  if (i < ntile_t * ntile_s) dtiles[i] = TileRef{0, (i / ntile_s) * TILE_TEST, (i % ntile_s) * TILE_SRC, 0};
}

}  // namespace sldm

extern "C" int sldm_kbar_noalloc(const sldm_mesh* m, int32_t obj, double k_re, double k_im, void* K_out, void* stream) {
  using namespace sldm;
  try {
    SLDM_REQUIRE(m && K_out, SLDM_EINVAL, "kbar_noalloc: null argument");
    SLDM_REQUIRE(obj >= 0 && obj < m->h.nobj, SLDM_EINVAL, "kbar_noalloc: object index out of range");
    SLDM_REQUIRE(std::isfinite(k_re) && std::isfinite(k_im), SLDM_EINVAL, "kbar_noalloc: non-finite wavenumber");
    int dev = 0;
    SLDM_CUDA(cudaGetDevice(&dev));
    SLDM_REQUIRE(dev == m->device, SLDM_EINVAL, "kbar_noalloc: current device differs from the mesh's device");
    const HostMesh& h = m->h;
    const int t0 = h.tri_begin[obj], nt_o = h.tri_begin[obj + 1] - t0;
    const int e0 = h.edge_begin[obj], ne_o = h.edge_begin[obj + 1] - e0;
    const int b0 = h.bedge_begin[obj], nbe_o = h.bedge_begin[obj + 1] - b0;
    const int ntile_t = (nt_o + TILE_TEST - 1) / TILE_TEST, ntile_s = (6 * nt_o + TILE_SRC - 1) / TILE_SRC;
    const size_t nkb = size_t(ne_o) * size_t(nbe_o);
    SLDM_REQUIRE(nkb <= NOALLOC_MAX_KB && size_t(ntile_t) * ntile_s <= NOALLOC_MAX_TILES, SLDM_EINVAL,
                 "kbar_noalloc: object too large for the fixed scratch (edges x barycentric edges = " +
                     std::to_string(nkb) + " > " + std::to_string(NOALLOC_MAX_KB) + ")");
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = static_cast<unsigned char*>(noalloc_scratch(dev));
    KTask* dtask = reinterpret_cast<KTask*>(base + NOALLOC_TASK_OFF);
    TileRef* dtiles = reinterpret_cast<TileRef*>(base + NOALLOC_TILE_OFF);
    double2* Kb = reinterpret_cast<double2*>(base + NOALLOC_KB_OFF);
    KTask t{};
    t.t0 = t0; t.ntest = nt_o; t.c0 = 6 * t0; t.nsrc = 6 * nt_o;
    t.e_row0 = e0; t.b_col0 = b0; t.ld = nbe_o;
    t.Kb = Kb;
    t.kr = k_re; t.ki = k_im;
    SLDM_REQUIRE(!split_rules_K(h, t).split, SLDM_ENOTSUP,
                 "kbar_noalloc: the object's sources must be split for this wavenumber (good conductor); "
                 "sldm_assemble handles it");
    // the block accumulates atomically: it must start at zero on every call
    SLDM_CUDA(cudaMemsetAsync(Kb, 0, nkb * sizeof(double2), s));
    const int nset = ntile_t * ntile_s;
    noalloc_setup_kernel<<<(nset + 127) / 128, 128, 0, s>>>(t, ntile_t, ntile_s, dtask, dtiles), ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
    const DevMesh& d = m->d;
    fill_K_bulk<double><<<unsigned(nset), TILE_SRC, 0, s>>>(dtask, dtiles, d.geo.p, d.bgeo.p, d.tri.p, d.tri_edge.p,
                                                            d.btri_edge.p), ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
    const int np = int(h.touchK_a.size());
    if (np > 0)
      fill_K_touch_one<<<(np + 127) / 128, 128, 0, s>>>(t, d.touchK_a.p, d.touchK_c.p, np, d.geo.p, d.bgeo.p, d.xyz.p,
                                                        d.tri.p, d.tri_edge.p, d.btri_edge.p), ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
    contract_bc<double>(m, obj, Kb, nbe_o, K_out, ne_o, s);
  } catch (const sldm::Error& e) {
    sldm::set_error(e.msg);
    return e.code;
  } catch (const std::bad_alloc&) {
    sldm::set_error("kbar_noalloc: host allocation failed");
    return SLDM_ENOMEM;
  } catch (const std::exception& e) {
    sldm::set_error(e.what());
    return SLDM_EINVAL;
  }
  return SLDM_OK;
}
