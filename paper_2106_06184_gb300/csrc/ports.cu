// Delta-gap edge ports (Sec. IV-B: a delta-gap edge port at the centre of the
// dipole, where S11 is measured; Sec. IV-C: two ports on the inductor).
//
// A port is the ring of edges of one object that lie in a plane s . r = c with
// one triangle on each side; an edge's sign is +1 when its T+ lies on the -s
// side (the RWG's unit flux crosses the plane along +s).  The source is an
// impressed field V delta(s . r - c) s on the surface, which enters the
// external EFIE as an incident field does: tested with the unit-flux RWGs it
// is sign V on the ring edges and zero elsewhere, b = sign V / eta0 in the
// system's scaling.  The port current is the electric surface current n x H
// through the ring along +s, I = sum sign j / (j k0) over the ring (j = j k0 H).
#include <cmath>
#include <complex>
#include <vector>

#include "internal.h"

namespace sldm {

namespace {

__device__ __forceinline__ int port_of(const int32_t* __restrict__ ptr, int nports, int e) {
  int p = 0;
  while (p + 1 < nports && ptr[p + 1] <= e) ++p;
  return p;
}

// b[:, k] += sum_p V[p, k] port_p / eta0.  Grid (ring entries / 128, ncols).
__global__ void port_rhs_kernel(int nports, const int32_t* __restrict__ ptr, const int32_t* __restrict__ edges,
                                const int8_t* __restrict__ signs, const double2* __restrict__ V, double inv_eta0,
                                double2* __restrict__ b, int64_t ldb) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (e >= ptr[nports]) return;
  const int p = port_of(ptr, nports, e);
  const double2 v = V[p + int64_t(nports) * k];
  const double sg = double(signs[e]) * inv_eta0;
  double2* d = b + int64_t(k) * ldb + edges[e];
  atomicAdd(&d->x, sg * v.x);  // a ring edge may belong to more than one port
  atomicAdd(&d->y, sg * v.y);
}

// I[p, k] = sum over ring p of sign x[edge, k] / (j k0).  Block per (port, column).
__global__ void port_currents_kernel(int nports, const int32_t* __restrict__ ptr, const int32_t* __restrict__ edges,
                                     const int8_t* __restrict__ signs, const double2* __restrict__ x, int64_t ldx,
                                     double k0, double2* __restrict__ I) {
  __shared__ double sr[32], si[32];
  const int p = blockIdx.x, k = blockIdx.y;
  double ar = 0.0, ai = 0.0;
  for (int e = ptr[p] + threadIdx.x; e < ptr[p + 1]; e += blockDim.x) {
    const double2 v = x[int64_t(k) * ldx + edges[e]];
    ar += double(signs[e]) * v.x;
    ai += double(signs[e]) * v.y;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_xor_sync(0xffffffffu, ar, o);
    ai += __shfl_xor_sync(0xffffffffu, ai, o);
  }
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    sr[w] = ar;
    si[w] = ai;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tr = 0.0, ti = 0.0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      tr += sr[i];
      ti += si[i];
    }
    I[p + int64_t(nports) * k] = make_double2(ti / k0, -tr / k0);  // (tr + j ti) / (j k0)
  }
}

}  // namespace

void port_check(const HostMesh& h, int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs) {
  SLDM_REQUIRE(nports >= 1 && ring_ptr && edges && signs, SLDM_EINVAL, "ports: invalid arguments");
  SLDM_REQUIRE(ring_ptr[0] == 0, SLDM_EINVAL, "ports: ring_ptr[0] must be 0");
  for (int p = 0; p < nports; ++p)
    SLDM_REQUIRE(ring_ptr[p + 1] > ring_ptr[p], SLDM_EINVAL, "ports: every port needs at least one edge");
  for (int e = 0; e < ring_ptr[nports]; ++e) {
    SLDM_REQUIRE(edges[e] >= 0 && edges[e] < h.ne, SLDM_EINVAL, "ports: edge index out of range");
    SLDM_REQUIRE(signs[e] == 1 || signs[e] == -1, SLDM_EINVAL, "ports: edge signs must be +1 or -1");
  }
}

void port_rhs(int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs, const double2* V,
              int32_t ncols, double2* b, int64_t ldb, cudaStream_t s) {
  const int ntot = ring_ptr[nports];
  DBuf<int32_t> dp, de;
  DBuf<int8_t> ds;
  DBuf<double2> dv;
  dp.upload(std::vector<int32_t>(ring_ptr, ring_ptr + nports + 1), s);
  de.upload(std::vector<int32_t>(edges, edges + ntot), s);
  ds.upload(std::vector<int8_t>(signs, signs + ntot), s);
  dv.upload(std::vector<double2>(V, V + size_t(nports) * ncols), s);
  const double eta0 = 4e-7 * 3.14159265358979323846 * 299792458.0;  // mu0 c0
  port_rhs_kernel<<<dim3(unsigned((ntot + 127) / 128), unsigned(ncols)), 128, 0, s>>>(nports, dp.p, de.p, ds.p, dv.p,
                                                                                   1.0 / eta0, b, ldb);
  count_launch();
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaStreamSynchronize(s));  // the uploads are freed on return
}

void port_currents(int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs, const double2* x,
                   int64_t ldx, int32_t ncols, double k0, double2* I_host, cudaStream_t s) {
  const int ntot = ring_ptr[nports];
  DBuf<int32_t> dp, de;
  DBuf<int8_t> ds;
  DBuf<double2> di;
  dp.upload(std::vector<int32_t>(ring_ptr, ring_ptr + nports + 1), s);
  de.upload(std::vector<int32_t>(edges, edges + ntot), s);
  ds.upload(std::vector<int8_t>(signs, signs + ntot), s);
  di.alloc(size_t(nports) * ncols);
  port_currents_kernel<<<dim3(unsigned(nports), unsigned(ncols)), 128, 0, s>>>(nports, dp.p, de.p, ds.p, x, ldx, k0, di.p);
  count_launch();
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaMemcpyAsync(I_host, di.p, size_t(nports) * ncols * sizeof(double2), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
}

}  // namespace sldm

using namespace sldm;

extern "C" {

int sldm_port_ring(const sldm_mesh* m, int32_t obj, const double* s, double c, double tol, int32_t cap, int32_t* edges,
                   int8_t* signs, int32_t* count) {
  try {
    SLDM_REQUIRE(m && s && count && cap >= 0 && (cap == 0 || (edges && signs)), SLDM_EINVAL, "port_ring: invalid arguments");
    const HostMesh& h = m->h;
    SLDM_REQUIRE(obj >= 0 && obj < h.nobj, SLDM_EINVAL, "port_ring: object index out of range");
    const double sn = std::sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
    SLDM_REQUIRE(sn > 0 && std::isfinite(sn), SLDM_EINVAL, "port_ring: the plane normal must be a nonzero vector");
    const double u[3] = {s[0] / sn, s[1] / sn, s[2] / sn};
    if (!(tol > 0)) {
      double ext = 0;
      for (int d = 0; d < 3; ++d) {
        double lo = 1e300, hi = -1e300;
        for (int64_t v = 0; v < h.nv; ++v) {
          lo = std::min(lo, h.xyz[3 * v + d]);
          hi = std::max(hi, h.xyz[3 * v + d]);
        }
        ext = std::max(ext, hi - lo);
      }
      tol = 1e-9 * ext;
    }
    auto dist = [&](int64_t v) { return h.xyz[3 * v] * u[0] + h.xyz[3 * v + 1] * u[1] + h.xyz[3 * v + 2] * u[2] - c; };
    auto cen = [&](int32_t t) {
      return (dist(h.tri[3 * t]) + dist(h.tri[3 * t + 1]) + dist(h.tri[3 * t + 2])) / 3.0;
    };
    int32_t n = 0;
    for (int32_t e = h.edge_begin[obj]; e < h.edge_begin[obj + 1]; ++e) {
      if (std::fabs(dist(h.uv[2 * e])) > tol || std::fabs(dist(h.uv[2 * e + 1])) > tol) continue;
      const double cp = cen(h.tplus[e]), cm = cen(h.tminus[e]);
      if (!(cp * cm < 0)) continue;  // both triangles on one side of the plane
      if (n < cap) {
        edges[n] = e;
        signs[n] = cp < 0 ? 1 : -1;
      }
      ++n;
    }
    *count = n;
    SLDM_REQUIRE(n > 0, SLDM_EINVAL, "port_ring: no edge of the object lies in the port plane");
    SLDM_REQUIRE(n <= cap, SLDM_EINVAL, "port_ring: capacity below the ring's size (see *count)");
    return SLDM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return SLDM_EINVAL;
  }
}

int sldm_port_sparams(int32_t n, const double* Y, double z0, double* S) {
  try {
    SLDM_REQUIRE(n >= 1 && Y && S && z0 > 0 && std::isfinite(z0), SLDM_EINVAL, "port_sparams: invalid arguments");
    typedef std::complex<double> cd;
    // S (1 + z0 Y) = 1 - z0 Y, solved as (1 + z0 Y)^T S^T = (1 - z0 Y)^T by Gauss-Jordan with partial pivoting
    std::vector<cd> A(size_t(n) * n), B(size_t(n) * n);  // row-major A = (1 + z0 Y)^T, B = (1 - z0 Y)^T
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const cd y(Y[2 * (i + size_t(n) * j)], Y[2 * (i + size_t(n) * j) + 1]);  // Y[i, j], column-major
        const cd d = (i == j) ? cd(1.0) : cd(0.0);
        A[size_t(j) * n + i] = d + z0 * y;
        B[size_t(j) * n + i] = d - z0 * y;
      }
    // singular when a pivot falls to rounding level of the operands 1 and z0 Y
    double ymax = 0;
    for (int i = 0; i < 2 * n * n; i += 2) ymax = std::max(ymax, std::hypot(Y[i], Y[i + 1]));
    const double scale = 1.0 + z0 * ymax;
    for (int c = 0; c < n; ++c) {
      int piv = c;
      for (int r = c + 1; r < n; ++r)
        if (std::abs(A[size_t(r) * n + c]) > std::abs(A[size_t(piv) * n + c])) piv = r;
      SLDM_REQUIRE(std::abs(A[size_t(piv) * n + c]) > 1e-14 * scale, SLDM_ENUMERIC, "port_sparams: 1 + z0 Y is singular");
      if (piv != c)
        for (int j = 0; j < n; ++j) {
          std::swap(A[size_t(piv) * n + j], A[size_t(c) * n + j]);
          std::swap(B[size_t(piv) * n + j], B[size_t(c) * n + j]);
        }
      const cd inv = 1.0 / A[size_t(c) * n + c];
      for (int j = 0; j < n; ++j) {
        A[size_t(c) * n + j] *= inv;
        B[size_t(c) * n + j] *= inv;
      }
      for (int r = 0; r < n; ++r) {
        if (r == c) continue;
        const cd f = A[size_t(r) * n + c];
        if (f == cd(0.0)) continue;
        for (int j = 0; j < n; ++j) {
          A[size_t(r) * n + j] -= f * A[size_t(c) * n + j];
          B[size_t(r) * n + j] -= f * B[size_t(c) * n + j];
        }
      }
    }
    // B now holds S^T row-major: S[i, j] = B[j n + i]
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const cd v = B[size_t(j) * n + i];  // (S^T)[j, i] = S[i, j]
        S[2 * (i + size_t(n) * j)] = v.real();
        S[2 * (i + size_t(n) * j) + 1] = v.imag();
      }
    return SLDM_OK;
  } catch (const Error& e) {
    set_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    set_error(e.what());
    return SLDM_EINVAL;
  }
}

}  // extern "C"
