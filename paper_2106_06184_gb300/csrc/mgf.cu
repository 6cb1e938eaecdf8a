// Layered-medium Green's function of the external problem (Sec. II-C; Sec. IV:
// quasistatic part extracted and added back analytically, Sommerfeld integrals
// of the rest tabulated and interpolated), for source and observation points in
// one layer l of a stratified background.
//
// Mixed-potential kernels (normalised like the paper's operators: L^A_m uses
// G^A/mu0, L^phi_m uses eps0 K^phi), spectral form from transmission-line
// Green's functions of the TM (e) and TE (h) lines of layer l:
//   g_xx = V_i^h/(j w mu0),  k_phi = eps0 (j w/k_rho^2)(V_i^e - V_i^h),
//   g_zz = [mu_r (k_rho^2 - k_z^2)/(eps k_rho^2) I_v^e + (w^2 mu mu_r/k_rho^2) I_v^h]/(j w),
//   g_zu = j (mu_r/k_rho)(I_i^e - I_i^h),  g_uz = j (mu_r/k_rho)(V_v^e - V_v^h),
// spatial: S0 for xx, phi, zz and -j S1 for z-rho, rho-z (S_n[f] = 1/(2 pi) int f J_n k dk).
// The direct term (homogeneous kernel of layer l) is filled by the homogeneous
// path; the quasistatic images of the two adjacent interfaces are evaluated in
// closed form here; the remainder is A(rho, z + z') + B(rho, z - z') from two
// sets of 2-D tables (256 log-spaced rho x 128), bilinear in (log rho, .).
#include <algorithm>
#include <cmath>
#include <complex>

#include "dense.h"
#include "fill_dev.cuh"
#include "mgf.h"

namespace sldm {

// ---------------------------------------------------------------- complex FP64 helpers
struct cx {
  double r, i;
};
__host__ __device__ __forceinline__ cx mk(double r, double i = 0.0) { return {r, i}; }
__host__ __device__ __forceinline__ cx operator+(cx a, cx b) { return {a.r + b.r, a.i + b.i}; }
__host__ __device__ __forceinline__ cx operator-(cx a, cx b) { return {a.r - b.r, a.i - b.i}; }
__host__ __device__ __forceinline__ cx operator-(cx a) { return {-a.r, -a.i}; }
__host__ __device__ __forceinline__ cx operator*(cx a, cx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__host__ __device__ __forceinline__ cx operator*(double s, cx a) { return {s * a.r, s * a.i}; }
__host__ __device__ __forceinline__ cx operator*(cx a, double s) { return {s * a.r, s * a.i}; }
__host__ __device__ __forceinline__ cx operator/(cx a, cx b) {
  const double d = b.r * b.r + b.i * b.i;
  return {(a.r * b.r + a.i * b.i) / d, (a.i * b.r - a.r * b.i) / d};
}
__device__ __forceinline__ cx cexp_(cx a) {
  double s, c;
  sincos(a.i, &s, &c);
  const double e = exp(a.r);
  return {e * c, e * s};
}
// exp(-j k R) for complex k: exp(Im k R) (cos(Re k R) - j sin(Re k R)); no exp when k is real
__device__ __forceinline__ cx eikr(cx k, double R) {
  double s, c;
  sincos(k.r * R, &s, &c);
  if (k.i == 0.0) return {c, -s};
  const double e = exp(k.i * R);
  return {e * c, -e * s};
}
// principal square root without cancellation: the larger of |Re|, |Im| comes
// from sqrt((|a| + |Re a|)/2), the other from Im a / (2 that)
__device__ __forceinline__ cx csqrt_(cx a) {
  if (a.r == 0.0 && a.i == 0.0) return {0.0, 0.0};
  const double t = sqrt(0.5 * (hypot(a.r, a.i) + fabs(a.r)));
  if (a.r >= 0.0) return {t, a.i / (2.0 * t)};
  return {fabs(a.i) / (2.0 * t), a.i < 0 ? -t : t};
}
// k_z = sqrt(k^2 - k_rho^2) with Im k_z <= 0
__device__ __forceinline__ cx kz_of(cx k, cx kr) {
  cx q = csqrt_(k * k - kr * kr);
  if (q.i > 0) q = -q;
  return q;
}

// J_n(z), n = 0, 1, complex z: periodic trapezoid rule of (1/2pi) int_0^2pi cos(n t - z sin t) dt
__device__ void bessel01_complex(cx z, cx* j0, cx* j1) {
  const double az = sqrt(z.r * z.r + z.i * z.i);
  const int M = 2 * (int(az) + 40);
  cx s0 = mk(0), s1 = mk(0);
  for (int m = 0; m < M; ++m) {
    double st, ct;
    sincospi(2.0 * m / M, &st, &ct);
    // cos(n t - z sin t) = (e^{i(nt - z st)} + e^{-i(nt - z st)})/2, z complex
    const cx ph = mk(z.r * st, z.i * st);  // z sin t
    // cos(w) for complex w = a + j b: cos a cosh b - j sin a sinh b
    auto ccos = [](cx w) {
      double sa, ca;
      sincos(w.r, &sa, &ca);
      if (w.i == 0.0) return cx{ca, 0.0};
      return cx{ca * cosh(w.i), -sa * sinh(w.i)};
    };
    s0 = s0 + ccos(-ph);
    // n = 1: cos(t - z sin t)
    const double t = 2.0 * M_PI * m / M;
    s1 = s1 + ccos(mk(t - ph.r, -ph.i));
  }
  *j0 = (1.0 / M) * s0;
  *j1 = (1.0 / M) * s1;
}

// ---------------------------------------------------------------- stack on the device
struct DevStack {
  int nl, l, pec, pad;
  double omega;
  cx eps[MGF_MAX_LAYERS];
  double mu[MGF_MAX_LAYERS];
  double d[MGF_MAX_LAYERS];  // thickness (finite layers)
  double zb, zu;             // bounds of layer l (+-1e300 for none)
  int top, bot;              // adjacent interfaces exist
};

constexpr double EPS0_ = 1.0 / (4e-7 * 3.14159265358979323846 * 299792458.0 * 299792458.0);
constexpr double MU0_ = 4e-7 * 3.14159265358979323846;
constexpr double C0_ = 299792458.0;

// generalised reflections (Gu, Gd) of line `te` (0 = e, 1 = h) seen from layer l
__device__ void reflections(const DevStack& S, cx kr, int te, cx* Gu, cx* Gd) {
  const double k0 = S.omega / C0_;
  cx Z[MGF_MAX_LAYERS], kz[MGF_MAX_LAYERS];
  for (int i = 0; i < S.nl; ++i) {
    // k_i = k0 sqrt(eps mu)
    cx k = csqrt_(S.mu[i] * S.eps[i]);
    k = k0 * k;
    kz[i] = kz_of(k, kr);
    Z[i] = te == 0 ? kz[i] / (S.omega * EPS0_ * S.eps[i]) : (S.omega * MU0_ * S.mu[i]) * (mk(1) / kz[i]);
  }
  auto fres = [&](int i, int j) { return (Z[j] - Z[i]) / (Z[j] + Z[i]); };
  cx up = mk(0);
  for (int i = 1; i <= S.l; ++i) {
    const cx f = fres(i, i - 1);
    if (i - 1 == 0) {
      up = f;
    } else {
      const cx ph = up * cexp_(mk(0, -2.0) * kz[i - 1] * mk(S.d[i - 1]));
      up = (f + ph) / (mk(1) + f * ph);
    }
  }
  const int last = S.nl - 1;
  cx down = S.pec ? mk(-1) : mk(0);
  for (int i = last - 1; i >= S.l; --i) {
    const cx f = fres(i, i + 1);
    if (i + 1 == last && !S.pec) {
      down = f;
    } else {
      const cx ph = down * cexp_(mk(0, -2.0) * kz[i + 1] * mk(S.d[i + 1]));
      down = (f + ph) / (mk(1) + f * ph);
    }
  }
  if (S.l == last) down = S.pec ? mk(-1) : mk(0);
  if (S.l == 0) up = mk(0);
  *Gu = up;
  *Gd = down;
}

// Remainder spectral kernels at one node: part 0 = single reflections minus the
// quasistatic images (argument s = z + z'), part 1 = double reflections (argument d = z - z').
__device__ void spectral_rem(const DevStack& S, const MgfStatic& Q, cx kr, int part, double arg, cx out[5]) {
  const double k0 = S.omega / C0_;
  const cx epsl = S.eps[S.l];
  const double mur = S.mu[S.l];
  cx k = k0 * csqrt_(mur * epsl);
  const cx kz = kz_of(k, kr);
  const cx Ze = kz / (S.omega * EPS0_ * epsl);
  const cx Zh = (S.omega * MU0_ * mur) * (mk(1) / kz);
  cx Gue, Gde, Guh, Gdh;
  reflections(S, kr, 0, &Gue, &Gde);
  reflections(S, kr, 1, &Guh, &Gdh);
  const double dl = S.zu - S.zb;
  const cx zero = mk(0);
  cx E1 = zero, E2 = zero, E3 = zero, E4 = zero;
  const cx mj = mk(0, -1);
  if (part == 0) {
    if (S.top) E1 = cexp_(mj * kz * mk(2 * S.zu - arg));
    if (S.bot) E2 = cexp_(mj * kz * mk(arg - 2 * S.zb));
  } else if (S.top && S.bot) {
    E3 = cexp_(mj * kz * mk(2 * dl + arg));
    E4 = cexp_(mj * kz * mk(2 * dl - arg));
  }
  const cx e2d = (S.top && S.bot) ? cexp_(mk(0, -2.0) * kz * mk(dl)) : zero;
  const cx De = mk(1) - Gue * Gde * e2d, Dh = mk(1) - Guh * Gdh * e2d;
  // reflected parts of the line functions
  auto Vi = [&](cx Z, cx Gu, cx Gd, cx D) { return (0.5 * Z) * ((Gu * E1 + Gd * E2 + Gu * Gd * (E3 + E4)) / D); };
  auto Iv = [&](cx Z, cx Gu, cx Gd, cx D) {
    return (mk(0.5) / Z) * ((-(Gu * E1) - Gd * E2 + Gu * Gd * (E3 + E4)) / D);
  };
  auto Ii = [&](cx Gu, cx Gd, cx D) { return 0.5 * ((-(Gu * E1) + Gd * E2 + Gu * Gd * (E3 - E4)) / D); };
  auto Vv = [&](cx Gu, cx Gd, cx D) { return 0.5 * ((Gu * E1 - Gd * E2 + Gu * Gd * (E3 - E4)) / D); };
  const cx Vie = Vi(Ze, Gue, Gde, De), Vih = Vi(Zh, Guh, Gdh, Dh);
  const cx Ive = Iv(Ze, Gue, Gde, De), Ivh = Iv(Zh, Guh, Gdh, Dh);
  const cx Iie = Ii(Gue, Gde, De), Iih = Ii(Guh, Gdh, Dh);
  const cx Vve = Vv(Gue, Gde, De), Vvh = Vv(Guh, Gdh, Dh);
  const cx jw = mk(0, S.omega);
  const cx kr2 = kr * kr;
  const cx gue = {Q.gue.r, Q.gue.i}, guh = {Q.guh.r, Q.guh.i}, gde = {Q.gde.r, Q.gde.i}, gdh = {Q.gdh.r, Q.gdh.i};
  out[0] = Vih / (jw * mk(MU0_));                                                    // xx
  out[1] = (EPS0_ * (jw / kr2)) * (Vie - Vih);                                        // phi
  out[2] = ((mur * ((kr2 - kz * kz) / (EPS0_ * epsl * kr2))) * Ive +
            ((S.omega * S.omega * MU0_ * mur * mur) * (mk(1) / kr2)) * Ivh) / jw;     // zz
  out[3] = (mk(0, mur) / kr) * (Iie - Iih);                                           // z-rho
  out[4] = (mk(0, mur) / kr) * (Vve - Vvh);                                           // rho-z
  if (part == 0) {
    const cx g = mk(1) / (mk(0, 2) * kz);
    out[0] = out[0] - (mur * (guh * E1 + gdh * E2)) * g;
    out[1] = out[1] - ((gue * E1 + gde * E2) * g) / epsl;
    out[2] = out[2] - (mur * ((guh - 2.0 * gue) * E1 + (gdh - 2.0 * gde) * E2)) * g;
    // z-rho / rho-z: the static single reflections exp(-k_rho zeta) (closed form in space: static_zr)
    const cx X1 = S.top ? cexp_(-(kr * mk(2 * S.zu - arg))) : zero;
    const cx X2 = S.bot ? cexp_(-(kr * mk(arg - 2 * S.zb))) : zero;
    const cx cu = gue - guh, cdn = gde - gdh;
    const cx c = mk(0, 0.5 * mur) / kr;
    out[3] = out[3] - c * (cdn * X2 - cu * X1);
    out[4] = out[4] - c * (cu * X1 - cdn * X2);
  }
}

// F[c][node][j] = w_node k_node g_c(k_node; arg_j) / (2 pi)
__global__ void mgf_spectral_kernel(DevStack S, MgfStatic Q, const double2* __restrict__ nodes,
                                    const double2* __restrict__ weights, int nnodes, const double* __restrict__ args,
                                    int nargs, int part, double2* F) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(nnodes) * nargs) return;
  const int n = int(idx / nargs), j = int(idx % nargs);
  const cx kr = {nodes[n].x, nodes[n].y};
  const cx w = {weights[n].x, weights[n].y};
  cx g[5];
  spectral_rem(S, Q, kr, part, args[j], g);
  const cx f = (0.5 / 3.14159265358979323846) * (w * kr);
  for (int c = 0; c < 5; ++c) {
    const cx v = f * g[c];
    F[(int64_t(c) * nnodes + n) * nargs + j] = make_double2(v.r, v.i);
  }
}

// Jm[order][i][n] = J_order(k_n rho_i)
__global__ void mgf_bessel_kernel(const double2* __restrict__ nodes, int nnodes, const double* __restrict__ rho, int nr,
                                  double2* Jm) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(nnodes) * nr) return;
  const int i = int(idx / nnodes), n = int(idx % nnodes);
  const double2 k = nodes[n];
  cx j0, j1;
  if (k.y == 0.0) {
    // real axis (the tail panels, arguments up to ~1e4): the math library's J0, J1
    j0 = mk(::j0(k.x * rho[i]));
    j1 = mk(::j1(k.x * rho[i]));
  } else {
    // the elliptic arc (|z| below ~1e2): the periodic trapezoid rule is accurate to
    // rounding once it has 2(|z| + 40) points
    bessel01_complex(mk(k.x * rho[i], k.y * rho[i]), &j0, &j1);
  }
  Jm[int64_t(i) * nnodes + n] = make_double2(j0.r, j0.i);
  Jm[int64_t(nr) * nnodes + int64_t(i) * nnodes + n] = make_double2(j1.r, j1.i);
}

// part[split][c][i][j] = sum over the split's nodes n of J_{order(c)}[i][n] F[c][n][j]:
// a complex product (rows i: rho, columns j: arguments) blocked as CT_I rows x 128
// columns per CTA, CT_N nodes of J staged in shared memory per step, the nodes
// split over gridDim.z / 5 CTAs (summed in a fixed order by mgf_sum_splits).
constexpr int CT_I = 8, CT_N = 32;
__global__ void __launch_bounds__(128) mgf_contract_kernel(const double2* __restrict__ Jm, const double2* __restrict__ F, int nnodes,
                                                           int nr, int nargs, int per_split, double2* part) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i0 = blockIdx.y * CT_I;
  const int c = blockIdx.z % 5, split = blockIdx.z / 5;
  const int order = c >= 3 ? 1 : 0;
  const double2* J = Jm + int64_t(order) * nr * nnodes;
  const double2* Fc = F + int64_t(c) * nnodes * nargs;
  const int n_begin = split * per_split, n_end = min(nnodes, n_begin + per_split);
  __shared__ double2 Js[CT_I][CT_N];
  cx acc[CT_I];
#pragma unroll
  for (int ii = 0; ii < CT_I; ++ii) acc[ii] = mk(0);
  for (int n0 = n_begin; n0 < n_end; n0 += CT_N) {
    for (int e = threadIdx.x; e < CT_I * CT_N; e += blockDim.x) {
      const int ii = e / CT_N, q = e % CT_N;
      const int gi = i0 + ii, gn = n0 + q;
      Js[ii][q] = (gi < nr && gn < n_end) ? J[int64_t(gi) * nnodes + gn] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (j < nargs) {
      const int nq = min(CT_N, n_end - n0);
      for (int q = 0; q < nq; ++q) {
        const double2 f = Fc[int64_t(n0 + q) * nargs + j];
#pragma unroll
        for (int ii = 0; ii < CT_I; ++ii) {
          const double2 a = Js[ii][q];
          acc[ii].r = fma(a.x, f.x, fma(-a.y, f.y, acc[ii].r));
          acc[ii].i = fma(a.x, f.y, fma(a.y, f.x, acc[ii].i));
        }
      }
    }
    __syncthreads();
  }
  if (j >= nargs) return;
  for (int ii = 0; ii < CT_I; ++ii)
    if (i0 + ii < nr) part[((int64_t(split) * 5 + c) * nr + i0 + ii) * nargs + j] = make_double2(acc[ii].r, acc[ii].i);
}

// table[c][i][j] = sum over splits of part (in split order), times -j for the order-1 components
__global__ void mgf_sum_splits(const double2* __restrict__ part, int nsplit, int64_t per, int nr, int nargs, double2* table) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= per) return;
  double re = 0, im = 0;
  for (int sp = 0; sp < nsplit; ++sp) {
    const double2 v = part[int64_t(sp) * per + idx];
    re += v.x;
    im += v.y;
  }
  const int c = int(idx / (int64_t(nr) * nargs));
  table[idx] = c >= 3 ? make_double2(im, -re) : make_double2(re, im);
}

// ---------------------------------------------------------------- host: nodes and tables
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p1 = 1.0, p2 = 0.0;
      for (int j = 1; j <= n; ++j) {
        const double p3 = p2;
        p2 = p1;
        p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
      }
      const double pp = n * (z * p1 - p2) / (z * z - 1.0);
      const double z1 = z;
      z = z1 - p1 / pp;
      if (std::fabs(z - z1) < 1e-16) {
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
        break;
      }
      x[i] = -z;
      w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
  }
}

// Elliptic arc k(t) = a/2 (1 - cos t) + j b sin t over t in [0, pi] (n_e Gauss points),
// a = max(1.5 max Re k_i, 2 k0), b = min(a/2, 2/rho_max); then Gauss-Legendre panels
// (16 points) of width min(pi/rho_max, (k_end - a)/4) up to k_end = a + 32/zeta_min.
static void sommerfeld_nodes(const MgfStackHost& H, double omega, double rho_max, double zeta_min,
                             std::vector<double2>& nodes, std::vector<double2>& weights) {
  const double k0 = omega / C0_;
  double kmax = 0;
  for (size_t i = 0; i < H.eps.size(); ++i) kmax = std::max(kmax, std::abs((k0 * std::sqrt(H.eps[i] * H.mu[i])).real()));
  const double a = std::max(1.5 * kmax, 2.0 * k0);
  const double b = std::min(0.5 * a, 2.0 / rho_max);
  std::vector<double> x, w;
  gauss_legendre(MGF_N_ELLIPSE, x, w);
  nodes.clear();
  weights.clear();
  for (int i = 0; i < MGF_N_ELLIPSE; ++i) {
    const double t = 0.5 * M_PI * (x[i] + 1), wt = 0.5 * M_PI * w[i];
    nodes.push_back(make_double2(0.5 * a * (1 - std::cos(t)), b * std::sin(t)));
    weights.push_back(make_double2(0.5 * a * std::sin(t) * wt, b * std::cos(t) * wt));
  }
  const double kend = a + 32.0 / zeta_min;
  const double width = std::min(M_PI / rho_max, (kend - a) / 4);
  const int npan = int(std::ceil((kend - a) / width));
  gauss_legendre(MGF_PER_PANEL, x, w);
  for (int p = 0; p < npan; ++p) {
    const double mid = a + width * (p + 0.5);
    for (int q = 0; q < MGF_PER_PANEL; ++q) {
      nodes.push_back(make_double2(mid + 0.5 * width * x[q], 0.0));
      weights.push_back(make_double2(0.5 * width * w[q], 0.0));
    }
  }
}

static DevStack dev_stack(const MgfStackHost& H, double omega) {
  DevStack S{};
  S.nl = int(H.eps.size());
  S.l = H.l;
  S.pec = H.pec;
  S.omega = omega;
  for (int i = 0; i < S.nl; ++i) {
    S.eps[i] = {H.eps[i].real(), H.eps[i].imag()};
    S.mu[i] = H.mu[i];
    S.d[i] = H.d[i];
  }
  S.zb = H.zb;
  S.zu = H.zu;
  S.top = H.top;
  S.bot = H.bot;
  return S;
}

static void build_one(const MgfStackHost& H, const MgfStatic& Q, double omega, const std::vector<double>& rho,
                      const std::vector<double>& args, int part, double zeta_min, double2* out, cudaStream_t s) {
  std::vector<double2> nodes, weights;
  sommerfeld_nodes(H, omega, rho.back() / 1.0, zeta_min, nodes, weights);
  const int nn = int(nodes.size()), nr = int(rho.size()), na = int(args.size());
  DBuf<double2> dn, dw, F, Jm;
  DBuf<double> dr, da;
  dn.upload(nodes, s);
  dw.upload(weights, s);
  dr.upload(rho, s);
  da.upload(args, s);
  F.alloc(size_t(nn) * na * 5);
  Jm.alloc(size_t(2) * nr * nn);
  const DevStack S = dev_stack(H, omega);
  {
    ScopedTimer tm("mgf_tables", s);
    const int64_t tot = int64_t(nn) * na;
    mgf_spectral_kernel<<<unsigned((tot + 127) / 128), 128, 0, s>>>(S, Q, dn.p, dw.p, nn, da.p, na, part, F.p), ::sldm::count_launch();
    const int64_t totb = int64_t(nn) * nr;
    mgf_bessel_kernel<<<unsigned((totb + 127) / 128), 128, 0, s>>>(dn.p, nn, dr.p, nr, Jm.p), ::sldm::count_launch();
    // split the nodes so that the product runs ~4 CTAs per SM
    const int base = ((na + 127) / 128) * ((nr + CT_I - 1) / CT_I) * 5;
    const int nsplit = std::max(1, std::min(64, (4 * 152 + base - 1) / base));
    const int per_split = ((nn + nsplit - 1) / nsplit + CT_N - 1) / CT_N * CT_N;
    const int64_t per = int64_t(5) * nr * na;
    DBuf<double2> part;
    part.alloc(size_t(nsplit) * per);
    mgf_contract_kernel<<<dim3((na + 127) / 128, (nr + CT_I - 1) / CT_I, 5 * nsplit), 128, 0, s>>>(Jm.p, F.p, nn, nr, na,
                                                                                                   per_split, part.p),
        ::sldm::count_launch();
    mgf_sum_splits<<<unsigned((per + 255) / 256), 256, 0, s>>>(part.p, nsplit, per, nr, na, out), ::sldm::count_launch();
    SLDM_CUDA(cudaStreamSynchronize(s));
  }
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaStreamSynchronize(s));
}

void mgf_build_tables(const MgfStackHost& H, double omega, double rho_min, double rho_max, double zmin, double zmax,
                      MgfTables& T, cudaStream_t s) {
  T.nr = MGF_NR;
  T.ns = MGF_NS;
  T.nd = MGF_ND;
  std::vector<double> rho(T.nr), sv(T.ns), dv(T.nd);
  for (int i = 0; i < T.nr; ++i)
    rho[i] = std::exp(std::log(rho_min) + (std::log(rho_max) - std::log(rho_min)) * i / (T.nr - 1));
  for (int j = 0; j < T.ns; ++j) sv[j] = 2 * zmin + (2 * zmax - 2 * zmin) * j / (T.ns - 1);
  for (int j = 0; j < T.nd; ++j) dv[j] = (zmax - zmin) * j / (T.nd - 1);
  T.lr0 = std::log(rho_min);
  T.lr1 = std::log(rho_max);
  T.s0 = 2 * zmin;
  T.s1 = 2 * zmax;
  T.d1 = zmax - zmin;
  T.A.alloc(size_t(5) * T.nr * T.ns);
  T.B.alloc(size_t(5) * T.nr * T.nd);
  // Objects may rest on an interface, where z + z' - 2 z_b = 0 and nothing decays
  // exponentially: the Sommerfeld tail is cut where exp(-k_rho zeta_floor) < 1e-14,
  // zeta_floor = 1/16 of the objects' height (the remainder decays algebraically
  // once every static image is out).
  const double zfloor = zmax > zmin ? (zmax - zmin) / 16 : 1e-3 * rho_max;
  double zeta_a = 1.0;
  {
    bool any = false;
    double zm = 1e300;
    if (H.top) {
      zm = std::min(zm, 2 * H.zu - 2 * zmax);
      any = true;
    }
    if (H.bot) {
      zm = std::min(zm, 2 * zmin - 2 * H.zb);
      any = true;
    }
    if (any) zeta_a = std::max(zm, zfloor);
  }
  build_one(H, T.Q, omega, rho, sv, 0, zeta_a, T.A.p, s);
  T.hasB = H.top && H.bot;
  if (H.top && H.bot) {
    const double zeta_b = std::max(2 * (H.zu - H.zb) - (zmax - zmin), zfloor);
    build_one(H, T.Q, omega, rho, dv, 1, zeta_b, T.B.p, s);
  } else {
    T.B.zero(s);
  }
}

// ---------------------------------------------------------------- reflected fill of L^A_m, L^phi_m
struct TabView {
  const double2* A;
  const double2* B;
  int nr, ns, nd;
  double lr0, lr1, s0, s1, d1;
  int hasB;
  double rmin, inv_rmin;  // exp(lr0), exp(-lr0)
  double sx, ss, sd;      // index scales (nr - 1)/(lr1 - lr0), (ns - 1)/(s1 - s0), (nd - 1)/d1 (0 if d1 = 0)
};

// Bilinear cell of a table at fractional indices (fx, fy), clamped as bilin does.
struct Cell {
  int64_t i00, i10, i01, i11;
  double w00, w10, w01, w11;
};
__device__ __forceinline__ Cell cell(int nr, int ny, double fx, double fy) {
  fx = fmin(fmax(fx, 0.0), nr - 1 - 1e-9);
  fy = ny > 1 ? fmin(fmax(fy, 0.0), ny - 1 - 1e-9) : 0.0;
  const int ix = int(fx), iy = int(fy);
  const double tx = fx - ix, ty = fy - iy;
  const int iy1 = min(iy + 1, ny - 1);
  return {int64_t(ix) * ny + iy, int64_t(ix + 1) * ny + iy, int64_t(ix) * ny + iy1, int64_t(ix + 1) * ny + iy1,
          (1 - tx) * (1 - ty), tx * (1 - ty), (1 - tx) * ty, tx * ty};
}
__device__ __forceinline__ cx at(const double2* t, int64_t plane, const Cell& c, int comp) {
  const double2* b = t + comp * plane;
  const double2 a00 = b[c.i00], a10 = b[c.i10], a01 = b[c.i01], a11 = b[c.i11];
  return {c.w00 * a00.x + c.w10 * a10.x + c.w01 * a01.x + c.w11 * a11.x,
          c.w00 * a00.y + c.w10 * a10.y + c.w01 * a01.y + c.w11 * a11.y};
}


// Static z-rho image in space: rho / (4 pi R (R + zeta)), R = |(rho, zeta)|, zeta >= 0; 0 at R = 0.
__device__ __forceinline__ double static_zr(double rho, double zeta) {
  const double R = sqrt(rho * rho + zeta * zeta);
  const double den = R * (R + zeta);
  return den > 0 ? (0.25 / 3.14159265358979323846) * rho / den : 0.0;
}

// Pair (t, s) touches through an interface when the triangles share a vertex on
// it: bits 0-2 (bottom) and 4-6 (top) of onmask flag vertices on the interfaces.
__device__ __forceinline__ bool touch_through(const int32_t* tri, int t, int s, int mt, int ms, int shift) {
  if (!((mt >> shift) & 7) || !((ms >> shift) & 7)) return false;
  for (int i = 0; i < 3; ++i) {
    if (!((mt >> (shift + i)) & 1)) continue;
    for (int j = 0; j < 3; ++j)
      if (((ms >> (shift + j)) & 1) && tri[3 * t + i] == tri[3 * s + j]) return true;
  }
  return false;
}

// One thread per (test, source) triangle pair of a block task, 6 x 6 points: the
// images (spherical waves and static z-rho / rho-z) and the tabulated remainder.
// An interface's images are left out for pairs touching through it (they are
// integrated apart by fill_reflected_touch); a coincident image point adds 0.
template <class C>
__global__ void __launch_bounds__(128) fill_reflected_kernel(const RTask* __restrict__ tasks, const double* __restrict__ geo,
                                                             const int32_t* __restrict__ tri_edge, const int32_t* __restrict__ tri,
                                                             const int32_t* __restrict__ onmask, DevStack S, MgfStatic Q, TabView T,
                                                             C* LA, int64_t ldA, C* LP, int64_t ldP) {
  const RTask tk = tasks[blockIdx.y];
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= int64_t(tk.ntest) * tk.nsrc) return;
  const int t = tk.t0 + int(p / tk.nsrc), sidx = tk.s0 + int(p % tk.nsrc);
  const double* gt = geo + size_t(t) * GEO_STRIDE;
  const double* gs = geo + size_t(sidx) * GEO_STRIDE;
  const double k0 = S.omega / C0_;
  const cx epsl = S.eps[S.l];
  const double mur = S.mu[S.l];
  const cx k = k0 * csqrt_(mur * epsl);
  const int mt = onmask[t], ms = onmask[sidx];
  const double use_bot = touch_through(tri, t, sidx, mt, ms, 0) ? 0.0 : 1.0;
  const double use_top = touch_through(tri, t, sidx, mt, ms, 4) ? 0.0 : 1.0;
  const cx gue = {Q.gue.r, Q.gue.i}, guh = {Q.guh.r, Q.guh.i}, gde = {Q.gde.r, Q.gde.i}, gdh = {Q.gdh.r, Q.gdh.i};
  const cx cu = gue - guh, cdn = gde - gdh;
  // image coefficients: xx mu_r g_h, phi g_e / eps_r, zz mu_r (g_h - 2 g_e), up and down
  const cx kxx_u = mur * guh, kxx_d = mur * gdh, kph_u = gue / epsl, kph_d = gde / epsl;
  const cx kzz_u = mur * (guh - 2.0 * gue), kzz_d = mur * (gdh - 2.0 * gde);
  cx loc[9];
  for (int i = 0; i < 9; ++i) loc[i] = mk(0);
  cx lp = mk(0);
  const double inv4pi = 0.25 / 3.14159265358979323846;
  for (int q = 0; q < 6; ++q) {
    double r[3], f[3][3];
    for (int d = 0; d < 3; ++d) r[d] = gt[GEO_C + d] + gt[GEO_RHO + 3 * q + d];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) f[i][d] = gt[GEO_SIG + i] * (gt[GEO_RHO + 3 * q + d] + gt[GEO_AV + 3 * i + d]);
    // Moments of the dyadic kernel T over the source points (weights w, offsets
    // rho_s from the source centre, rhohat = (hx, hy)): with f_j(r_s) = sig_j (rho_s + av_j),
    // sum_s w T . f_j = sig_j (M1 + M0 . av_j), T . u = (gxx u_x + grz hx u_z,
    // gxx u_y + grz hy u_z, gzz u_z + gzr (hx u_x + hy u_y)).
    cx a0 = mk(0), az = mk(0), bx = mk(0), by = mk(0), cxm = mk(0), cym = mk(0);      // M0
    cx a0x = mk(0), a0y = mk(0), bxz = mk(0), byz = mk(0), azz = mk(0), cr = mk(0);  // M1
    cx sphi = mk(0);
    for (int sq = 0; sq < 6; ++sq) {
      double rs[3];
      for (int d = 0; d < 3; ++d) rs[d] = gs[GEO_C + d] + gs[GEO_RHO + 3 * sq + d];
      const double dx = r[0] - rs[0], dy = r[1] - rs[1];
      const double rho2 = dx * dx + dy * dy;
      const double irho = rho2 > 0 ? rsqrt(rho2) : 0.0;
      const double rho = rho2 * irho;
      const double zz = r[2], zp = rs[2];
      // quasistatic images: spherical waves exp(-j k R)/(4 pi R) and the static
      // z-rho image rho / (4 pi R (R + zeta)) from the image points
      cx G1 = mk(0), G2 = mk(0);
      double F1 = 0, F2 = 0;
      if (S.top) {
        const double zeta = 2 * S.zu - zz - zp;
        const double R2 = rho2 + zeta * zeta;
        if (R2 > 0) {
          const double r1 = rsqrt(R2), R = R2 * r1;
          const double iR = use_top * inv4pi * r1;
          G1 = iR * eikr(k, R);
          F1 = iR * rho / (R + zeta);
        }
      }
      if (S.bot) {
        const double zeta = zz + zp - 2 * S.zb;
        const double R2 = rho2 + zeta * zeta;
        if (R2 > 0) {
          const double r1 = rsqrt(R2), R = R2 * r1;
          const double iR = use_bot * inv4pi * r1;
          G2 = iR * eikr(k, R);
          F2 = iR * rho / (R + zeta);
        }
      }
      cx gxx = kxx_u * G1 + kxx_d * G2;
      cx gphi = kph_u * G1 + kph_d * G2;
      cx gzz = kzz_u * G1 + kzz_d * G2;
      // tabulated remainder (one bilinear cell for the five components)
      const double lr = log(fmax(rho, T.rmin));
      const double fx = (lr - T.lr0) * T.sx;
      const double fs = (zz + zp - T.s0) * T.ss;
      const Cell ca = cell(T.nr, T.ns, fx, fs);
      const int64_t pa = int64_t(T.nr) * T.ns;
      gxx = gxx + at(T.A, pa, ca, 0);
      gphi = gphi + at(T.A, pa, ca, 1);
      gzz = gzz + at(T.A, pa, ca, 2);
      cx bzr = at(T.A, pa, ca, 3), brz = at(T.A, pa, ca, 4);
      const double dd = zz - zp;
      const double sg = dd > 0 ? 1.0 : (dd < 0 ? -1.0 : 0.0);
      if (T.hasB) {
        const double fd = fabs(dd) * T.sd;
        const Cell cb = cell(T.nr, T.nd, fx, fd);
        const int64_t pb = int64_t(T.nr) * T.nd;
        gxx = gxx + at(T.B, pb, cb, 0);
        gphi = gphi + at(T.B, pb, cb, 1);
        gzz = gzz + at(T.B, pb, cb, 2);
        bzr = bzr + sg * at(T.B, pb, cb, 3);
        brz = brz + sg * at(T.B, pb, cb, 4);
      }
      // the S1 (z-rho, rho-z) remainders vanish linearly at rho = 0: below rho_min scale by rho / rho_min
      const double lin = fmin(rho * T.inv_rmin, 1.0);
      const cx gzr = lin * bzr + mur * (cdn * F2 - cu * F1);
      const cx grz = lin * brz + mur * (cu * F1 - cdn * F2);
      const double hx = dx * irho, hy = dy * irho;
      const double w = gs[GEO_W + sq];
      const double px = gs[GEO_RHO + 3 * sq], py = gs[GEO_RHO + 3 * sq + 1], pz = gs[GEO_RHO + 3 * sq + 2];
      const cx wxx = w * gxx, wzz = w * gzz, wrx = (w * hx) * grz, wry = (w * hy) * grz;
      const cx wzx = (w * hx) * gzr, wzy = (w * hy) * gzr;
      a0 = a0 + wxx;
      az = az + wzz;
      bx = bx + wrx;
      by = by + wry;
      cxm = cxm + wzx;
      cym = cym + wzy;
      a0x = a0x + px * wxx;
      a0y = a0y + py * wxx;
      bxz = bxz + pz * wrx;
      byz = byz + pz * wry;
      azz = azz + pz * wzz;
      cr = cr + (px * wzx + py * wzy);
      sphi = sphi + w * gphi;
    }
    cx V[3][3];  // sum_s W' T . f_j(r'_s)
    for (int j = 0; j < 3; ++j) {
      const double sj = gs[GEO_SIG + j];
      const double ux = gs[GEO_AV + 3 * j], uy = gs[GEO_AV + 3 * j + 1], uz = gs[GEO_AV + 3 * j + 2];
      V[j][0] = sj * (a0x + ux * a0 + bxz + uz * bx);
      V[j][1] = sj * (a0y + uy * a0 + byz + uz * by);
      V[j][2] = sj * (azz + uz * az + cr + ux * cxm + uy * cym);
    }
    const double wq = gt[GEO_W + q];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) loc[3 * i + j] = loc[3 * i + j] + wq * (f[i][0] * V[j][0] + f[i][1] * V[j][1] + f[i][2] * V[j][2]);
    lp = lp + wq * sphi;
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C* dst = LA + int64_t(tri_edge[3 * t + i]) * ldA + tri_edge[3 * sidx + j];
      if (sizeof(dst->x) == 4) {
        atomicAdd(reinterpret_cast<float2*>(dst), make_float2(float(loc[3 * i + j].r), float(loc[3 * i + j].i)));
      } else {
        atomicAdd(reinterpret_cast<double*>(dst), loc[3 * i + j].r);
        atomicAdd(reinterpret_cast<double*>(dst) + 1, loc[3 * i + j].i);
      }
    }
  const double sc = 1.0 / (gt[GEO_A] * gs[GEO_A]);
  C* dp = LP + int64_t(t) * ldP + sidx;
  dp->x = decltype(dp->x)(double(dp->x) + sc * lp.r);
  dp->y = decltype(dp->y)(double(dp->y) + sc * lp.i);
}

// ---------------------------------------------------------------- pairs touching through an interface
// Gauss-Legendre nodes and weights on [0, 1] of the Duffy rule
static __constant__ double c_duffy_x[MGF_DUFFY_N], c_duffy_w[MGF_DUFFY_N];

// The point of triangle (a, b, c) nearest to r: the projection on the plane when
// inside, else the nearest point of the three edges.
__device__ void closest_point(const double* r, const double* a, const double* b, const double* c, double* out) {
  double v0[3], v1[3], n[3];
  for (int d = 0; d < 3; ++d) {
    v0[d] = b[d] - a[d];
    v1[d] = c[d] - a[d];
  }
  n[0] = v0[1] * v1[2] - v0[2] * v1[1];
  n[1] = v0[2] * v1[0] - v0[0] * v1[2];
  n[2] = v0[0] * v1[1] - v0[1] * v1[0];
  const double nn = n[0] * n[0] + n[1] * n[1] + n[2] * n[2];
  const double h = ((r[0] - a[0]) * n[0] + (r[1] - a[1]) * n[1] + (r[2] - a[2]) * n[2]) / nn;
  double p[3], v2[3];
  for (int d = 0; d < 3; ++d) {
    p[d] = r[d] - h * n[d];
    v2[d] = p[d] - a[d];
  }
  const double d00 = v0[0] * v0[0] + v0[1] * v0[1] + v0[2] * v0[2];
  const double d01 = v0[0] * v1[0] + v0[1] * v1[1] + v0[2] * v1[2];
  const double d11 = v1[0] * v1[0] + v1[1] * v1[1] + v1[2] * v1[2];
  const double d20 = v2[0] * v0[0] + v2[1] * v0[1] + v2[2] * v0[2];
  const double d21 = v2[0] * v1[0] + v2[1] * v1[1] + v2[2] * v1[2];
  const double den = d00 * d11 - d01 * d01;
  const double bv = (d11 * d20 - d01 * d21) / den, bw = (d00 * d21 - d01 * d20) / den;
  if (bv >= 0 && bw >= 0 && bv + bw <= 1) {
    for (int d = 0; d < 3; ++d) out[d] = p[d];
    return;
  }
  const double* E[4] = {a, b, c, a};
  double best = 1e300;
  for (int e = 0; e < 3; ++e) {
    const double* u = E[e];
    const double* v = E[e + 1];
    double uv[3], ur[3];
    for (int d = 0; d < 3; ++d) {
      uv[d] = v[d] - u[d];
      ur[d] = r[d] - u[d];
    }
    double t = (ur[0] * uv[0] + ur[1] * uv[1] + ur[2] * uv[2]) / (uv[0] * uv[0] + uv[1] * uv[1] + uv[2] * uv[2]);
    t = fmin(fmax(t, 0.0), 1.0);
    double qd[3], dist = 0;
    for (int d = 0; d < 3; ++d) {
      qd[d] = u[d] + t * uv[d];
      dist += (r[d] - qd[d]) * (r[d] - qd[d]);
    }
    dist = sqrt(dist);
    if (dist < best) {
      best = dist;
      for (int d = 0; d < 3; ++d) out[d] = qd[d];
    }
  }
}

// One group of 8 threads per pair touching through an interface (thread q < 6:
// outer point q of the test triangle): that interface's images over the mirrored
// source triangle (x', y', 2 z_I - z'), where the RWG keeps its transverse part and
// flips its z part.  xx, phi, zz: the spherical wave with 1/R and R in closed form
// over the mirrored triangle and the rest by its 6 points; z-rho, rho-z: the static
// kernel (r - r'')_t / (4 pi R (R + zeta)) by the Duffy rule (n x n Gauss points on
// each of the three parts of the mirrored triangle split at its point nearest r).
template <class C>
__global__ void fill_reflected_touch(const int32_t* __restrict__ pairs, int npairs, const double* __restrict__ geo,
                                     const double* __restrict__ xyz, const int32_t* __restrict__ tri,
                                     const int32_t* __restrict__ tri_edge, DevStack S, MgfStatic Q, C* LA, int64_t ldA, C* LP,
                                     int64_t ldP) {
  const int64_t gt_ = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int p = int(gt_ >> 3), q = int(gt_ & 7);
  const bool valid = p < npairs;
  const int t = valid ? pairs[3 * p] : 0, sidx = valid ? pairs[3 * p + 1] : 0, top = valid ? pairs[3 * p + 2] : 0;
  const bool act = valid && q < 6;
  double m[20];
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = 0.0;
  const double* gt = geo + size_t(t) * GEO_STRIDE;
  const double* gs = geo + size_t(sidx) * GEO_STRIDE;
  if (act) {
    const double k0 = S.omega / C0_;
    const cx epsl = S.eps[S.l];
    const double mur = S.mu[S.l];
    const cx k = k0 * csqrt_(mur * epsl);
    const cx k2 = k * k;
    const double zI = top ? S.zu : S.zb;
    const cx ge = top ? cx{Q.gue.r, Q.gue.i} : cx{Q.gde.r, Q.gde.i};
    const cx gh = top ? cx{Q.guh.r, Q.guh.i} : cx{Q.gdh.r, Q.gdh.i};
    const cx czr = top ? -(mur * (ge - gh)) : mur * (ge - gh), crz = -czr;
    const cx cxx = mur * gh, czz = mur * (gh - 2.0 * ge), cphi = ge / epsl;
    double Bm[3][3];  // mirrored source vertices
    for (int j = 0; j < 3; ++j)
      for (int d = 0; d < 3; ++d) Bm[j][d] = d == 2 ? 2 * zI - xyz[3 * tri[3 * sidx + j] + 2] : xyz[3 * tri[3 * sidx + j] + d];
    double r[3], f[3][3];
    for (int d = 0; d < 3; ++d) r[d] = gt[GEO_C + d] + gt[GEO_RHO + 3 * q + d];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) f[i][d] = gt[GEO_SIG + i] * (gt[GEO_RHO + 3 * q + d] + gt[GEO_AV + 3 * i + d]);
    // int G and int p G over the mirrored triangle
    cx I0 = mk(0), Ip[3] = {mk(0), mk(0), mk(0)};
    for (int j = 0; j < 6; ++j) {
      double rs[3];
      for (int d = 0; d < 3; ++d) rs[d] = gs[GEO_C + d] + gs[GEO_RHO + 3 * j + d];
      rs[2] = 2 * zI - rs[2];
      const double dx = r[0] - rs[0], dy = r[1] - rs[1], dz = r[2] - rs[2];
      const cd g = green_smooth(cd{k.r, k.i}, sqrt(dx * dx + dy * dy + dz * dz));
      const double w = gs[GEO_W + j];
      I0 = I0 + w * cx{g.r, g.i};
      for (int d = 0; d < 3; ++d) Ip[d] = Ip[d] + (w * rs[d]) * cx{g.r, g.i};
    }
    Pot P;
    potentials(r, Bm[0], Bm[1], Bm[2], P);
    I0 = I0 + mk(INV4PI * P.inv_r) - (0.5 * INV4PI * P.r) * k2;
    for (int d = 0; d < 3; ++d)
      Ip[d] = Ip[d] + mk(INV4PI * (P.por[d] + P.rho[d] * P.inv_r)) - (0.5 * INV4PI * (P.pr[d] + P.rho[d] * P.r)) * k2;
    // static z-rho kernel by the Duffy rule: J0 = int W, J1[d][e] = int W_d p_e
    double J0[2] = {0, 0}, J1[2][3] = {{0, 0, 0}, {0, 0, 0}};
    {
      double Qp[3];
      closest_point(r, Bm[0], Bm[1], Bm[2], Qp);
      double e1[3], e2[3];
      for (int d = 0; d < 3; ++d) {
        e1[d] = Bm[1][d] - Bm[0][d];
        e2[d] = Bm[2][d] - Bm[0][d];
      }
      const double fx_ = e1[1] * e2[2] - e1[2] * e2[1], fy_ = e1[2] * e2[0] - e1[0] * e2[2], fz_ = e1[0] * e2[1] - e1[1] * e2[0];
      const double full = sqrt(fx_ * fx_ + fy_ * fy_ + fz_ * fz_);
      for (int sub = 0; sub < 3; ++sub) {
        const double* P1 = Bm[sub];
        const double* P2 = Bm[(sub + 1) % 3];
        double a1[3], a2v[3];
        for (int d = 0; d < 3; ++d) {
          a1[d] = P1[d] - Qp[d];
          a2v[d] = P2[d] - P1[d];
        }
        const double cx_ = a1[1] * a2v[2] - a1[2] * a2v[1], cy_ = a1[2] * a2v[0] - a1[0] * a2v[2],
                     cz_ = a1[0] * a2v[1] - a1[1] * a2v[0];
        const double a2 = sqrt(cx_ * cx_ + cy_ * cy_ + cz_ * cz_);
        if (a2 <= 1e-12 * full) continue;
        for (int iu = 0; iu < MGF_DUFFY_N; ++iu) {
          const double u = c_duffy_x[iu];
          for (int iv = 0; iv < MGF_DUFFY_N; ++iv) {
            const double v = c_duffy_x[iv];
            const double wt = a2 * u * c_duffy_w[iu] * c_duffy_w[iv];
            double pt[3];
            for (int d = 0; d < 3; ++d) pt[d] = Qp[d] + u * a1[d] + u * v * a2v[d];
            const double dx = r[0] - pt[0], dy = r[1] - pt[1], dz = r[2] - pt[2];
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double den = R * (R + fabs(dz));
            if (!(den > 0)) continue;
            const double s_ = wt * INV4PI / den;
            const double wx = s_ * dx, wy = s_ * dy;
            J0[0] += wx;
            J0[1] += wy;
            for (int e = 0; e < 3; ++e) {
              J1[0][e] += wx * pt[e];
              J1[1][e] += wy * pt[e];
            }
          }
        }
      }
    }
    const double wq = gt[GEO_W + q];
    for (int j = 0; j < 3; ++j) {
      const double sb = gs[GEO_SIG + j];
      cx in[3];
      for (int d = 0; d < 3; ++d) in[d] = Ip[d] - Bm[j][d] * I0;  // int (p'' - v''_j) G
      const double tj = (J1[0][0] - Bm[j][0] * J0[0]) + (J1[1][1] - Bm[j][1] * J0[1]);
      const double zj0 = J1[0][2] - Bm[j][2] * J0[0], zj1 = J1[1][2] - Bm[j][2] * J0[1];
      for (int i = 0; i < 3; ++i) {
        const cx v = (wq * sb) * (cxx * (f[i][0] * in[0] + f[i][1] * in[1]) - czz * (f[i][2] * in[2]) +
                                  czr * (f[i][2] * tj) - crz * (f[i][0] * zj0 + f[i][1] * zj1));
        m[2 * (3 * i + j)] = v.r;
        m[2 * (3 * i + j) + 1] = v.i;
      }
    }
    const cx l = (wq / (gt[GEO_A] * gs[GEO_A])) * (cphi * I0);
    m[18] = l.r;
    m[19] = l.i;
  }
#pragma unroll
  for (int i = 0; i < 20; ++i) m[i] = grp_sum8(m[i]);
  if (!valid || q != 0) return;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      C* dst = LA + int64_t(tri_edge[3 * t + i]) * ldA + tri_edge[3 * sidx + j];
      if (sizeof(dst->x) == 4) {
        atomicAdd(reinterpret_cast<float2*>(dst), make_float2(float(m[2 * (3 * i + j)]), float(m[2 * (3 * i + j) + 1])));
      } else {
        atomicAdd(reinterpret_cast<double*>(dst), m[2 * (3 * i + j)]);
        atomicAdd(reinterpret_cast<double*>(dst) + 1, m[2 * (3 * i + j) + 1]);
      }
    }
  C* dp = LP + int64_t(t) * ldP + sidx;
  if (sizeof(dp->x) == 4) {
    atomicAdd(reinterpret_cast<float2*>(dp), make_float2(float(m[18]), float(m[19])));
  } else {
    atomicAdd(reinterpret_cast<double*>(dp), m[18]);
    atomicAdd(reinterpret_cast<double*>(dp) + 1, m[19]);
  }
}

// Per triangle: bits 0-2 / 4-6 flag vertices on the bottom / top interface of the
// objects' layer (to 1e-9 of the mesh size); the pairs touching through an
// interface among the listed blocks (t, s, 0 = bottom / 1 = top).
void mgf_touch_setup(const HostMesh& h, const MgfStackHost& H, const std::vector<RTask>& tasks, std::vector<int32_t>& onmask,
                     std::vector<int32_t>& pairs) {
  double span = 0;
  for (int d = 0; d < 3; ++d) {
    double a = 1e300, b = -1e300;
    for (int64_t v = 0; v < h.nv; ++v) {
      a = std::min(a, h.xyz[3 * v + d]);
      b = std::max(b, h.xyz[3 * v + d]);
    }
    span = std::max(span, b - a);
  }
  const double tol = 1e-9 * span;
  onmask.assign(h.nt, 0);
  std::vector<int32_t> touching;
  for (int64_t t = 0; t < h.nt; ++t) {
    int msk = 0;
    for (int i = 0; i < 3; ++i) {
      const double z = h.xyz[3 * size_t(h.tri[3 * t + i]) + 2];
      if (H.bot && std::fabs(z - H.zb) <= tol) msk |= 1 << i;
      if (H.top && std::fabs(z - H.zu) <= tol) msk |= 1 << (4 + i);
    }
    onmask[t] = msk;
    if (msk) touching.push_back(int32_t(t));
  }
  pairs.clear();
  // `touching` is sorted: each task's test and source ranges are two slices of it
  auto slice = [&](int32_t lo, int32_t n) {
    return std::make_pair(std::lower_bound(touching.begin(), touching.end(), lo),
                          std::lower_bound(touching.begin(), touching.end(), lo + n));
  };
  for (const RTask& k : tasks) {
    const auto ta = slice(k.t0, k.ntest), tb = slice(k.s0, k.nsrc);
    for (auto ia = ta.first; ia != ta.second; ++ia) {
      const int32_t a = *ia;
      for (auto ib = tb.first; ib != tb.second; ++ib) {
        const int32_t b = *ib;
        for (int plane = 0; plane < 2; ++plane) {
          const int sh = plane ? 4 : 0;
          bool hit = false;
          for (int i = 0; i < 3 && !hit; ++i)
            for (int j = 0; j < 3 && !hit; ++j)
              hit = ((onmask[a] >> (sh + i)) & 1) && ((onmask[b] >> (sh + j)) & 1) && h.tri[3 * size_t(a) + i] == h.tri[3 * size_t(b) + j];
          if (hit) {
            pairs.push_back(a);
            pairs.push_back(b);
            pairs.push_back(plane);
          }
        }
      }
    }
  }
}

template <class C>
void mgf_fill_reflected(const sldm_mesh* m, const MgfStackHost& H, double omega, const MgfTables& T,
                        const std::vector<RTask>& tasks, void* LA, int64_t ldA, void* LP, int64_t ldP, cudaStream_t s) {
  if (tasks.empty()) return;
  const DevStack S = dev_stack(H, omega);
  TabView tv{T.A.p, T.B.p, T.nr, T.ns, T.nd, T.lr0, T.lr1, T.s0, T.s1, T.d1, T.hasB ? 1 : 0, std::exp(T.lr0), std::exp(-T.lr0),
             (T.nr - 1) / (T.lr1 - T.lr0), T.s1 > T.s0 ? (T.ns - 1) / (T.s1 - T.s0) : 0.0, T.d1 > 0 ? (T.nd - 1) / T.d1 : 0.0};
  ScopedTimer tm("fill_reflected", s);
  std::vector<int32_t> onmask, pairs;
  mgf_touch_setup(m->h, H, tasks, onmask, pairs);
  DBuf<RTask> dt;
  DBuf<int32_t> dm, dp;
  dt.upload(tasks, s);
  dm.upload(onmask, s);
  int64_t most = 0;
  double pairs_total = 0;
  for (const RTask& k : tasks) {
    most = std::max(most, int64_t(k.ntest) * k.nsrc);
    pairs_total += double(k.ntest) * k.nsrc;
  }
  {
    ScopedTimer tb("fill_reflected_bulk", s);
    timer_units("fill_reflected_bulk", 36.0 * pairs_total);
    fill_reflected_kernel<C><<<dim3(unsigned((most + 127) / 128), unsigned(tasks.size())), 128, 0, s>>>(
        dt.p, m->d.geo.p, m->d.tri_edge.p, m->d.tri.p, dm.p, S, T.Q, tv, (C*)LA, ldA, (C*)LP, ldP), ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
  }
  const int np = int(pairs.size() / 3);
  if (np > 0) {
    std::vector<double> x, w;
    gauss_legendre(MGF_DUFFY_N, x, w);
    for (int i = 0; i < MGF_DUFFY_N; ++i) {
      x[i] = 0.5 * (x[i] + 1);
      w[i] = 0.5 * w[i];
    }
    SLDM_CUDA(cudaMemcpyToSymbol(c_duffy_x, x.data(), sizeof(double) * MGF_DUFFY_N));
    SLDM_CUDA(cudaMemcpyToSymbol(c_duffy_w, w.data(), sizeof(double) * MGF_DUFFY_N));
    dp.upload(pairs, s);
    const int64_t threads = int64_t(np) * 8;
    fill_reflected_touch<C><<<unsigned((threads + 127) / 128), 128, 0, s>>>(dp.p, np, m->d.geo.p, m->d.xyz.p, m->d.tri.p,
                                                                            m->d.tri_edge.p, S, T.Q, (C*)LA, ldA, (C*)LP, ldP),
        ::sldm::count_launch();
    SLDM_CUDA(cudaGetLastError());
  }
  // the uploads above are released at scope exit: finish their readers first
  SLDM_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------- stack helpers (host)
MgfStatic mgf_static(const MgfStackHost& H) {
  MgfStatic Q{};
  const int L = int(H.eps.size()), l = H.l;
  const std::complex<double> el = H.eps[l];
  const double ml = H.mu[l];
  auto pair = [&](int j, std::complex<double>* ge, double* gh) {
    *ge = (el - H.eps[j]) / (el + H.eps[j]);
    *gh = (H.mu[j] - ml) / (H.mu[j] + ml);
  };
  std::complex<double> gue = 0, gde = 0;
  double guh = 0, gdh = 0;
  if (l > 0) pair(l - 1, &gue, &guh);
  if (l < L - 1) pair(l + 1, &gde, &gdh);
  else if (H.pec) {
    gde = -1.0;
    gdh = -1.0;
  }
  Q.gue = {gue.real(), gue.imag()};
  Q.gde = {gde.real(), gde.imag()};
  Q.guh = {guh, 0.0};
  Q.gdh = {gdh, 0.0};
  return Q;
}

// Normal-incidence plane wave through the stack: E_x = a e^{+j k (z - zref)} + c e^{-j k (z - zref)} in layer l.
// Oblique plane wave through the stack, incident from the upper half-space.  The
// transverse wavevector kt = k0 (khat_x, khat_y) is common to all layers; with
// rho = kt / |kt| (at normal incidence the transverse direction of pol) and
// phi = z x rho the field splits into TE (E along phi, line impedance
// w mu0 mu_i / k_z,i) and TM (H along phi, impedance k_z,i / (w eps0 eps_i)).  For each,
// the transverse E is a transmission line in z: in layer i it is
// a e^{+j k_z (z - zref)} + c e^{-j k_z (z - zref)}, c / a at the layer's bottom the
// reflection coefficient looking down, continuous across every interface.  In the
// objects' layer E = e^{-j kt.r} [phi V_TE + rho V_TM + z (|kt| / k_z)(a_TM e^+ - c_TM e^-)].
void mgf_plane_wave(const MgfStackHost& H, const std::vector<double>& thick, double z_top, double omega, const double* khat,
                    const double* pol, double rec[PW_REC]) {
  typedef std::complex<double> C;
  const int L = int(H.eps.size());
  const double k0 = omega / C0_;
  const double ktx = k0 * khat[0], kty = k0 * khat[1];
  const double krho = std::hypot(ktx, kty);
  double rx, ry;
  if (krho > 1e-12 * k0) {
    rx = ktx / krho;
    ry = kty / krho;
  } else {
    const double n = std::hypot(pol[0], pol[1]);
    rx = n > 0 ? pol[0] / n : 1.0;
    ry = n > 0 ? pol[1] / n : 0.0;
  }
  const double px = -ry, py = rx;  // phi = z x rho
  std::vector<C> kz(L), Z(L), down(L);
  std::vector<bool> finite(L);
  for (int i = 0; i < L; ++i) {
    C q = std::sqrt(C(k0 * k0) * H.eps[i] * H.mu[i] - C(krho * krho));
    if (q.imag() > 0) q = -q;
    kz[i] = q;
    finite[i] = i > 0 && (H.pec || i < L - 1);
  }
  for (int pt = 0; pt < 2; ++pt) {  // 0: TE, 1: TM
    for (int i = 0; i < L; ++i)
      Z[i] = pt == 0 ? C(omega * MU0_ * H.mu[i]) / kz[i] : kz[i] / (omega * EPS0_ * H.eps[i]);
    down[L - 1] = H.pec ? C(-1) : C(0);
    for (int i = L - 2; i >= 0; --i) {
      const C f = (Z[i + 1] - Z[i]) / (Z[i + 1] + Z[i]);
      const C ph = finite[i + 1] ? down[i + 1] * std::exp(C(0, -2) * kz[i + 1] * thick[i + 1]) : C(0);
      down[i] = (f + ph) / (C(1) + f * ph);
    }
    const double v0 = pt == 0 ? pol[0] * px + pol[1] * py : pol[0] * rx + pol[1] * ry;
    C a = v0 * std::exp(C(0, 1) * kz[0] * z_top), c = a * down[0];
    C v = a + c;
    for (int i = 1; i <= H.l; ++i) {
      const C gtop = finite[i] ? down[i] * std::exp(C(0, -2) * kz[i] * thick[i]) : C(0);
      a = v / (C(1) + gtop);
      c = a * gtop;
      if (finite[i]) v = a * std::exp(C(0, -1) * kz[i] * thick[i]) + c * std::exp(C(0, 1) * kz[i] * thick[i]);
    }
    rec[PW_A + 4 * pt] = a.real();
    rec[PW_A + 4 * pt + 1] = a.imag();
    rec[PW_A + 4 * pt + 2] = c.real();
    rec[PW_A + 4 * pt + 3] = c.imag();
  }
  // at normal incidence pol.rho carries the whole wave, so the TM form holds with krho = 0
  rec[PW_KT] = ktx;
  rec[PW_KT + 1] = kty;
  rec[PW_RHO] = rx;
  rec[PW_RHO + 1] = ry;
  rec[PW_KZ] = kz[H.l].real();
  rec[PW_KZ + 1] = kz[H.l].imag();
  rec[PW_KRHO] = krho;
  rec[PW_ZREF] = H.l == 0 ? z_top : H.zu;
}

template void mgf_fill_reflected<float2>(const sldm_mesh*, const MgfStackHost&, double, const MgfTables&,
                                         const std::vector<RTask>&, void*, int64_t, void*, int64_t, cudaStream_t);
template void mgf_fill_reflected<double2>(const sldm_mesh*, const MgfStackHost&, double, const MgfTables&,
                                          const std::vector<RTask>&, void*, int64_t, void*, int64_t, cudaStream_t);

}  // namespace sldm
