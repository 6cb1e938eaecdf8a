// Internal declarations shared by the translation units of libsldm.
#pragma once

#include <cuda_runtime.h>
#include <cuComplex.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/sldm.h"

namespace sldm {

// ---------------------------------------------------------------- errors
void set_error(const std::string& msg);
struct Error {
  int code;
  std::string msg;
};
#define SLDM_CUDA(call)                                                                   \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw ::sldm::Error{SLDM_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)
#define SLDM_REQUIRE(cond, code, msg)                 \
  do {                                                \
    if (!(cond)) throw ::sldm::Error{(code), (msg)};  \
  } while (0)

// ---------------------------------------------------------------- kernel timers
// Optional CUDA-event timing of named launches (sldm_timers_enable).  When
// disabled, timer_begin/timer_end cost one branch.
bool timers_on();
// Mute (or unmute) the timers for the calling thread only: its launches are
// left out of every timed name (autotuning passes).
void timers_mute(bool m);
// Counts kernel launches made by the library (sldm_launch_count); called right
// after each launch statement.
void count_launch();
void timer_begin(const char* name, cudaStream_t s);
void timer_end(cudaStream_t s);
// adds the algorithmic units (bytes moved, kernel evaluations) of a timed launch
void timer_units(const char* name, double units);
struct ScopedTimer {
  cudaStream_t s;
  bool on;
  ScopedTimer(const char* name, cudaStream_t s_) : s(s_), on(timers_on()) {
    if (on) timer_begin(name, s);
  }
  ~ScopedTimer() {
    if (on) timer_end(s);
  }
};

// ---------------------------------------------------------------- device-memory budget
// Bytes held by every DBuf of the library (all devices) and the optional limit
// set by sldm_set_device_budget (0 = none).  budget_take throws SLDM_ENOMEM
// when the limit would be exceeded.
void budget_take(size_t bytes);
void budget_give(size_t bytes);
// Test injection (sldm_test_inject): consumes one pending LU stall, if any.
bool take_lu_stall();

// ---------------------------------------------------------------- device buffers
template <class T>
struct DBuf {
  T* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void release() {
    if (p) {
      cudaFree(p);
      budget_give(n * sizeof(T));
    }
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    budget_take(count * sizeof(T));
    cudaError_t e = cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      budget_give(count * sizeof(T));
      throw Error{SLDM_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed"};
    }
    n = count;
  }
  void upload(const std::vector<T>& h, cudaStream_t s = 0) {
    alloc(h.size());
    if (!h.empty()) SLDM_CUDA(cudaMemcpyAsync(p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s = 0) {
    if (n) SLDM_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  size_t bytes() const { return n * sizeof(T); }
};

// ---------------------------------------------------------------- mesh
// Host topology and its device copy.  Triangle-local index i names the vertex
// tri[t][i] and the edge opposite to it.
struct HostMesh {
  int64_t nv = 0, nt = 0, ne = 0, nobj = 0, nbe = 0;
  double ell = 1.0;                        // mean edge length: the length unit of the scaled solve
  std::vector<double> xyz;                 // nv*3
  std::vector<int32_t> tri;                // nt*3
  std::vector<int32_t> obj;                // nt
  std::vector<int32_t> tri_edge;           // nt*3 edge opposite local vertex i
  std::vector<int8_t> tri_sign;            // nt*3 (+1: this triangle is T+)
  std::vector<int64_t> uv;                 // ne*2
  std::vector<int32_t> tplus, tminus;      // ne
  std::vector<int32_t> tri_begin, edge_begin, bedge_begin;  // nobj+1 each
  // barycentric refinement: child c = 6 t + k; its edges
  std::vector<int32_t> btri_edge;          // 6nt*3 barycentric edge opposite child-local vertex j
  std::vector<int8_t> btri_sign;           // 6nt*3
  // BC coefficients, CSC by BC column n: rows are barycentric edges
  std::vector<int32_t> bc_ptr, bc_row;     // ne+1, nnz
  std::vector<double> bc_val;              // nnz
  // touching pairs (within an object): primal-primal and primal-child
  std::vector<int32_t> touchL_a, touchL_b; // pairs sharing a vertex (including self)
  std::vector<int32_t> touchK_a, touchK_c; // (test triangle, touching child), own children excluded
  // I_x sparsity: CSR rows = edges; each nonzero lists its contributions
  std::vector<int32_t> ix_ptr, ix_col;     // ne+1, nnz
  std::vector<int32_t> ixc_ptr;            // nnz+1
  std::vector<int32_t> ixc_tri, ixc_child, ixc_i, ixc_j;  // per contribution
  std::vector<double> ixc_coef;            // C coefficient of the barycentric edge in BC n
};

struct DevMesh {
  DBuf<double> xyz;
  DBuf<int32_t> tri, tri_edge, tplus, tminus, obj, q2t, tri_begin, edge_begin;
  DBuf<int8_t> tri_sign, btri_sign;
  DBuf<int32_t> btri_edge;
  DBuf<int32_t> bc_ptr, bc_row;
  DBuf<double> bc_val;
  DBuf<int32_t> touchL_a, touchL_b, touchK_a, touchK_c;
  DBuf<int32_t> ix_ptr, ix_col, ixc_ptr, ixc_tri, ixc_child, ixc_i, ixc_j;
  DBuf<double> ixc_coef;
  // geometry computed on the device (see fill.cu: geometry_kernel)
  DBuf<double> geo;   // per triangle: GEO_STRIDE doubles
  DBuf<double> bgeo;  // per child: BGEO_STRIDE doubles
};

// Per-triangle geometry record (doubles): centroid(3) area(1) normal(3)
// quad local points rho_q = r_q - c (18) weights W_q = w_q A (6) a_i = c - v_i (9)
// edge factors s_i/(2A) (3)
constexpr int GEO_C = 0, GEO_A = 3, GEO_N = 4, GEO_RHO = 7, GEO_W = 25, GEO_AV = 31, GEO_SIG = 40;
constexpr int GEO_STRIDE = 43;

void build_host_mesh(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt, const int32_t* obj,
                     HostMesh& hm);

}  // namespace sldm

struct sldm_mesh {
  sldm::HostMesh h;
  sldm::DevMesh d;
  int device = 0;
};

struct sldm_stack {
  std::vector<sldm_layer> layers;
  double z_top = 0;
  int32_t bottom = 0;
};

namespace sldm {

// ---------------------------------------------------------------- delta-gap ports (ports.cu)
// SLDM_EINVAL unless ring_ptr is a CSR of nports non-empty rings of valid edges with signs +-1.
void port_check(const HostMesh& h, int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs);
// b[:, k] += sum_p V[p + nports k] port_p / eta0 (b on the device, column stride ldb; the rest host arrays).
void port_rhs(int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs, const double2* V,
              int32_t ncols, double2* b, int64_t ldb, cudaStream_t s);
// I_host[p + nports k] = sum over ring p of sign x[edge, k] / (j k0) (x on the device).
void port_currents(int32_t nports, const int32_t* ring_ptr, const int32_t* edges, const int8_t* signs, const double2* x,
                   int64_t ldx, int32_t ncols, double k0, double2* I_host, cudaStream_t s);

// ---------------------------------------------------------------- fill (fill.cu)
void geometry(const HostMesh& hm, DevMesh& dm, cudaStream_t s);

// One fill task: triangles [t0, t0+nt_test) x [s0, s0+nt_src) of the same
// mesh, results scattered (atomically added) into row-major complex blocks.
struct LTask {
  int32_t t0, ntest, s0, nsrc;
  int32_t e_row0, e_col0;     // edge offsets subtracted from global edge ids
  int32_t t_row0, t_col0;     // triangle offsets
  int64_t ldA, ldP;           // leading dimensions
  void* A;                    // L^A destination (complex of the op precision) or null
  void* P;                    // L^phi destination or null
  double kr, ki;              // wavenumber
  double sAr, sAi, sPr, sPi;  // complex scale of L^A and L^phi
};
struct KTask {
  int32_t t0, ntest;          // primal test triangles
  int32_t c0, nsrc;           // children [c0, c0 + nsrc) = 6 * source triangles
  int32_t e_row0, b_col0;     // edge and barycentric-edge offsets
  int64_t ld;
  void* Kb;                   // barycentric Kbar destination, complex of op precision
  double kr, ki;
};

template <class R>
void fill_L(const sldm_mesh* m, const std::vector<LTask>& tasks, cudaStream_t s);
template <class R>
void fill_K(const sldm_mesh* m, const std::vector<KTask>& tasks, cudaStream_t s);

// Good-conductor fills (fill_sub.cu).  One point of a source's quadrature:
// barycentric coordinates with respect to the source triangle and its weight as
// a fraction of the source's area.
struct __align__(32) SrcPoint {
  double x, y, z, w;
};
// The quadrature of every source of a task that has at least one source to
// split (else split = false and nothing else is filled): source i's points are
// pts[off[i] .. off[i + 1]).
struct SplitRules {
  bool split = false;
  std::vector<int32_t> off;
  std::vector<SrcPoint> pts;
};
SplitRules split_rules_L(const HostMesh& h, const LTask& tk);
SplitRules split_rules_K(const HostMesh& h, const KTask& tk);
template <class R>
void fill_L_split_task(const sldm_mesh* m, const LTask& tk, const SplitRules& rules, cudaStream_t s);
template <class R>
void fill_K_split_task(const sldm_mesh* m, const KTask& tk, const SplitRules& rules, cudaStream_t s);
// Kbar (ne_o x ne_o, op precision) = Kb (ne_o x nbe_o) * C_o, plus beta * I_x/2 (dense add of Gram)
template <class R>
void contract_bc(const sldm_mesh* m, int obj, const void* Kb, int64_t ldKb, void* K, int64_t ldK,
                 cudaStream_t s);
// Gram matrix values for the CSR pattern ix_ptr/ix_col (double)
void gram_ix(const sldm_mesh* m, double* vals, cudaStream_t s);
// e_inc for nrhs plane waves into b (complex128, column-major N x nrhs, ld)
void rhs_planewave(const sldm_mesh* m, double k0, const double* khat_pol_dev, int nrhs, double2* b,
                   int64_t ld, cudaStream_t s);
// Plane wave through a stack, one record per right-hand side (filled by mgf_plane_wave):
// kt (x, y), rho (x, y), a_TE, c_TE, a_TM, c_TM (re, im), k_z (re, im), |kt|, zref.
constexpr int PW_KT = 0, PW_RHO = 2, PW_A = 4, PW_KZ = 12, PW_KRHO = 14, PW_ZREF = 15, PW_REC = 16;
// e_inc in the objects' layer of a stack for nrhs plane waves (records rec_dev, PW_REC doubles each)
void rhs_planewave_layered(const sldm_mesh* m, const double* rec_dev, int nrhs, double2* b, int64_t ld, cudaStream_t s);
// RCS above a stack: per angle the theta- and phi-polarised plane-wave records
// (2n records of PW_REC doubles, device) of waves arriving from the observation
// direction; jd: nr columns of complex128 RWG coefficients (stride ldj), rcs:
// n x nr (stride n), device
void farfield_layered(const sldm_mesh* m, const double2* jd, int64_t ldj, int nr, const double* rec_dev, int n, double* rcs,
                      cudaStream_t s);
// far field in free space: angles (theta, phi) pairs, device; jd, rcs as above
void farfield(const sldm_mesh* m, double k0, const double2* jd, int64_t ldj, int nr, const double* ang_dev, int n,
              double* rcs, cudaStream_t s);

}  // namespace sldm
