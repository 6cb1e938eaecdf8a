// Layered-medium Green's function tables and reflected fill (mgf.cu).
#pragma once
#include <complex>

#include "internal.h"

namespace sldm {

constexpr int MGF_MAX_LAYERS = 8;
constexpr int MGF_N_ELLIPSE = 400;  // Gauss points on the elliptic arc of the Sommerfeld path
constexpr int MGF_PER_PANEL = 16;   // Gauss points per real-axis panel
constexpr int MGF_NR = 256, MGF_NS = 128, MGF_ND = 128;

// Quasistatic (k_rho -> infinity) reflection coefficients of layer l: e (TM) and h (TE), up and down.
struct MgfStatic {
  struct {
    double r, i;
  } gue, guh, gde, gdh;
};

// Stack as seen from layer l at one frequency.
struct MgfStackHost {
  std::vector<std::complex<double>> eps;  // complex relative permittivity per layer
  std::vector<double> mu, d;              // relative permeability, thickness (finite layers)
  int l = 0, pec = 0;
  double zb = -1e300, zu = 1e300;         // bounds of layer l
  int top = 0, bot = 0;                   // interfaces above / below layer l exist
};

struct MgfTables {
  DBuf<double2> A, B;  // [5][nr][ns], [5][nr][nd]
  int nr = 0, ns = 0, nd = 0;
  bool hasB = false;   // double reflections (a layer with both interfaces)
  double lr0 = 0, lr1 = 0, s0 = 0, s1 = 0, d1 = 0;
  MgfStatic Q{};
};

MgfStatic mgf_static(const MgfStackHost& H);
void mgf_build_tables(const MgfStackHost& H, double omega, double rho_min, double rho_max, double zmin, double zmax,
                      MgfTables& T, cudaStream_t s);
// A block of the reflected fill: test triangles [t0, t0 + ntest) x sources [s0, s0 + nsrc).
struct RTask {
  int32_t t0, ntest, s0, nsrc;
};
constexpr int MGF_DUFFY_N = 16;  // Gauss points per direction of the Duffy rule on touching pairs
// Reflected part (images + tabulated remainder) of L^A_m, L^phi_m added over the
// listed blocks; pairs touching through an interface take that interface's
// images from the mirrored-triangle rules.
template <class C>
void mgf_fill_reflected(const sldm_mesh* m, const MgfStackHost& H, double omega, const MgfTables& T,
                        const std::vector<RTask>& tasks, void* LA, int64_t ldA, void* LP, int64_t ldP, cudaStream_t s);
// Per right-hand side record of a plane wave in the objects' layer (layout PW_*):
// kt (2), rho (2), a_TE, c_TE, a_TM, c_TM (complex), k_z (complex), |kt|, zref.
void mgf_plane_wave(const MgfStackHost& H, const std::vector<double>& thick, double z_top, double omega, const double* khat,
                    const double* pol, double rec[PW_REC]);

}  // namespace sldm
