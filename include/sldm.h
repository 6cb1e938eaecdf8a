/*
 * sldm.h - C ABI of the GB300 (sm_103a) implementation of the single-layer
 * dual-mesh boundary element method (SLDM-BEM) of Sharma & Triverio,
 * "A Single-Layer Dual-Mesh Boundary Element Method for Multiscale
 * Electromagnetic Modeling of Penetrable Objects in Layered Media",
 * arXiv:2106.06184.
 *
 * The library computes, on one GPU, the data-parallel hot path of the method:
 * the triangle-pair Gauss-quadrature fill of the single-layer operators L^(A),
 * L^(phi) and the double-layer operator Kbar (RWG testing on the primal mesh,
 * Buffa-Christiansen (BC) sources on its barycentric refinement) with
 * singularity extraction on touching pairs; the per-object admittance blocks
 * Y11, Y21 (Eq. Yeqdef); and the dense complex matrix-vector products of the
 * final system (Eq. finalsystem) that drive GMRES.
 *
 * General conventions
 *  - Every call returns an int status: SLDM_OK (0) or a negative SLDM_E* code;
 *    sldm_last_error() returns the text of the last error of the calling thread.
 *  - Handles are opaque, owned by the library, released by the matching
 *    *_destroy.  Caller arrays are borrowed for the duration of a call only.
 *  - Arrays passed with `where` = SLDM_HOST are host memory; with SLDM_DEVICE
 *    they are device memory on the device the handle was created on.
 *  - `stream` is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls that return results in host memory synchronise the stream.
 *  - Complex numbers are interleaved {re, im} pairs of double (complex128).
 *  - SI units; time convention exp(+j w t); G(R) = exp(-j k R)/(4 pi R) (Eq. hgf).
 *  - A handle may not be used by two threads at once; different handles may.
 *
 * Discretisation conventions (the paper defers D, B, F and the BC functions to
 * its references; these are the readings this library implements):
 *  - Triangles are given counter-clockwise seen from outside (outward normal);
 *    each object is a closed, oriented 2-manifold; objects are disjoint and
 *    occupy contiguous, non-decreasing obj_id ranges of the triangle list.
 *  - Edge n joins vertices u < v.  T+ is the triangle whose boundary runs
 *    u -> v, T- runs v -> u.  Edges are numbered by sorting (obj, u, v).
 *  - Area-normalised RWG f_n = (r - p+)/(2A+) on T+, -(r - p-)/(2A-) on T-
 *    (p = vertex opposite the edge): unit flux from T+ to T-.
 *  - Pulses h_p = 1/A_p; D[T+, n] = +1, D[T-, n] = -1.  Charge neutrality per
 *    object eliminates its last triangle: B = [I; -1^T], F = [I 0].
 *  - BC function of edge (u, v): unit flux from the dual cell of u to that of
 *    v, equal integrated divergence on the barycentric triangles of each cell,
 *    zero flux through the half edges u - m and v - m (b_n close to n x f_n).
 *  - Unknown vector (length N = 2 ne + nt - nobj), Eq. finalsystem:
 *        x = [ j k0 H (ne, RWG) ; E/eta0 (ne, BC, of n x E) ; -c0 rho (nt - nobj) ]
 *    where the charge entries skip each object's last triangle.
 *  - Final system rows: external EFIE (ne), internal EFIE (ne), external
 *    continuity (nt - nobj); row 2 carries -K with K = Kbar + I_x/2.
 */
#ifndef SLDM_H
#define SLDM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------- */
#define SLDM_OK 0
#define SLDM_EINVAL -1     /* invalid argument or mesh */
#define SLDM_ENOMEM -2     /* device/host allocation failed or budget exceeded */
#define SLDM_ENOTCONV -3   /* iterative solver did not reach the tolerance */
#define SLDM_ENUMERIC -4   /* NaN/Inf or a zero pivot */
#define SLDM_ECUDA -5      /* a CUDA runtime call failed */
#define SLDM_EBUSY -6      /* the handle is in use */
#define SLDM_ENOTSUP -7    /* feature not available in this build */
#define SLDM_ETIMEOUT -8   /* a bounded wait inside a kernel ran out (the context stays usable) */

#define SLDM_HOST 0
#define SLDM_DEVICE 1

#define SLDM_PREC_F64 0    /* complex128 operator, FP64 fill */
#define SLDM_PREC_F32 1    /* complex64 operator, FP32 bulk fill, FP64 singular terms */
/* complex64 operator with an FP64-accurate residual: every block is filled (and
 * Y11, Y21 factored) in FP64, then kept as two complex64 parts hi = fl32(v) and
 * lo = fl32(v - hi), so v = hi + lo to ~2^-48 relative.  GMRES cycles apply hi in
 * FP32 arithmetic; the residual of iterative refinement, and sldm_apply, apply
 * hi + lo with compensated FP32 sums (~48 bits), so refined solutions converge to
 * those of the FP64 discrete system.  Twice the operator memory of SLDM_PREC_F32
 * (the same as SLDM_PREC_F64). */
#define SLDM_PREC_F32X2 2

#define SLDM_BOTTOM_HALFSPACE 0
#define SLDM_BOTTOM_PEC 1

typedef struct sldm_mesh sldm_mesh;
typedef struct sldm_stack sldm_stack;
typedef struct sldm_op sldm_op;

/* Material of one object (Sec. II): relative permittivity, permeability,
 * conductivity (S/m) and the index of the background layer containing it. */
typedef struct {
  double eps_r, mu_r, sigma;
  int32_t layer;
  int32_t reserved;
} sldm_material;

/* One layer of the background, listed top to bottom.  The first layer is the
 * upper half-space; the last is the lower half-space unless the stack ends in
 * a PEC ground.  thickness is ignored for half-spaces. */
typedef struct {
  double eps_r, mu_r, sigma, thickness;
} sldm_layer;

typedef struct {
  int64_t nv, nt, ne, nobj;
  int64_t n_unknowns;   /* 2 ne + nt - nobj */
  int64_t n_bary_edges; /* 9 nt */
} sldm_mesh_info;

typedef struct {
  int32_t precision;    /* SLDM_PREC_F64, SLDM_PREC_F32 or SLDM_PREC_F32X2 */
  int32_t nested_min;   /* SLDM_PREC_F64 only: objects whose M_l has at least this order
                           (ne + nt - 1) get Y E by inner solves instead of a formed Y
                           (Sec. III: direct factorisation below ~1000 triangles): an
                           FP32 approximate inverse of M_l and FP64 iterative refinement
                           to 1e-13 per product; 0 = 2500, < 0 = always form Y.  Falls
                           back to the FP64 LU when the refinement would contract slowly. */
  void* stream;         /* stream the fill runs on (NULL = default) */
} sldm_assemble_opts;

#define SLDM_PRECOND_P 0     /* right preconditioner P of Eq. pcext (default) */
#define SLDM_PRECOND_NONE 1  /* no preconditioner */
#define SLDM_REFINE_AUTO 0   /* complex64 operators: FP64 residuals, iterative refinement (default) */
#define SLDM_REFINE_OFF 1    /* residuals in the operator's precision */

typedef struct {
  double tol;           /* relative residual of the length-scaled system (default 1e-8), see sldm_solve */
  int32_t restart;      /* GMRES restart length m (default 300; at most N and 1000) */
  int32_t maxit;        /* maximum iterations per right-hand side (default 2000) */
  int32_t x0_given;     /* nonzero: x holds the initial guess on entry */
  int32_t precond;      /* SLDM_PRECOND_P (0, default) or SLDM_PRECOND_NONE */
  int32_t refine;       /* SLDM_REFINE_AUTO (0, default) or SLDM_REFINE_OFF; see sldm_solve */
  int32_t reserved;
} sldm_solve_opts;

typedef struct {
  int32_t iters;        /* total GMRES iterations (over all right-hand sides) */
  int32_t status;       /* SLDM_OK or SLDM_ENOTCONV */
  double relres;        /* largest final relative residual over the right-hand sides */
} sldm_solve_info;

typedef struct {
  int64_t n_unknowns, ne, nt, nobj;
  int64_t device_bytes; /* device memory held by the operator */
  int32_t precision;
  int32_t tc_from;      /* complex64 operators: the smallest lockstep width whose
                           products run on the tensor cores (9, 17, or 33 = never),
                           chosen at assembly by timing both paths on the
                           operator's own blocks; 0 otherwise */
  double k0;
} sldm_op_info;

/* Operator blocks that sldm_op_block can copy out (for verification). */
#define SLDM_BLOCK_LAM 0    /* L^A_m  = mu_b L^A(k_b), ne x ne, global (Eq. AEFIEextdis) */
#define SLDM_BLOCK_LPM 1    /* L^phi_m = L^phi(k_b)/eps_b, nt x nt, global */
#define SLDM_BLOCK_LA 2     /* mu_r L^A(k), object, ne_o x ne_o (Eq. AEFIEintdis) */
#define SLDM_BLOCK_LP 3     /* L^phi(k)/eps_cr, object, nt_o x nt_o */
#define SLDM_BLOCK_K 4      /* K = Kbar(k) + I_x/2, object, ne_o x ne_o (Eq. Kmatdef) */
#define SLDM_BLOCK_Y11 5    /* Y11, object, ne_o x ne_o (Eq. Yeqdef) */
#define SLDM_BLOCK_Y21 6    /* Y21, object, (nt_o - 1) x ne_o */
#define SLDM_BLOCK_IX 7     /* I_x, dense copy of the sparse Gram matrix, ne x ne */
#define SLDM_BLOCK_KBAR_L 8 /* Kbar(k_l), object, ne_o x ne_o (equivalent configuration) */

/* Text of the last error of the calling thread, NUL-terminated, truncated to len. */
void sldm_last_error(char* buf, size_t len);

/* Build a mesh: topology (edges, T+/T-, barycentric refinement, BC
 * coefficients, touching-pair lists) on the host, then upload it to the
 * current device.  xyz: nv x 3 doubles; tri: nt x 3 vertex indices; obj_id: nt
 * non-decreasing object ids or NULL for one object.  Host pointers.
 * Errors: SLDM_EINVAL when an object is not a closed oriented manifold, is
 * oriented inward (its triangles' vertex order must be counter-clockwise seen
 * from outside: the formulation takes n as the outward normal, Sec. II), shares
 * a vertex with another object, a triangle is degenerate, or obj_id is not
 * contiguous.  These checks run on the host before any device call. */
int sldm_mesh_create(const double* xyz, int64_t nv, const int32_t* tri, int64_t nt,
                     const int32_t* obj_id, sldm_mesh** out);
int sldm_mesh_info_get(const sldm_mesh* mesh, sldm_mesh_info* info);
/* Edge table in the numbering above: uv (ne x 2), tplus, tminus (ne).  Host pointers; any may be NULL. */
int sldm_mesh_edges(const sldm_mesh* mesh, int64_t* uv, int64_t* tplus, int64_t* tminus);
int sldm_mesh_destroy(sldm_mesh* mesh);

/* Background medium (Sec. II, "stratified background").  nlayers == 1 with a
 * half-space bottom is a homogeneous background (L^A_m = mu_b L^A(k_b),
 * L^phi_m = L^phi(k_b)/eps_b).  Otherwise layers are listed top to bottom:
 * layer 0 is the upper half-space above z_top; each following layer is finite
 * (thickness > 0) except the last one when bottom = SLDM_BOTTOM_HALFSPACE; with
 * SLDM_BOTTOM_PEC a perfect conductor lies under the last layer.  At most 8 layers
 * (SLDM_ENOTSUP beyond); SLDM_EINVAL for non-positive or non-finite eps_r, mu_r, a
 * negative or non-finite sigma, a non-finite z_top or a finite layer without a
 * positive thickness (checked on the host, no device call).
 * In a stratified background every object lies inside one layer l
 * (sldm_material.layer, the same for all objects) and may rest on its interfaces
 * (vertices on an interface to 1e-9 of the mesh size), but none crosses one
 * (SLDM_EINVAL at assembly); the external operators use
 * the multilayer kernel of that layer (homogeneous kernel of layer l, quasistatic
 * images of the adjacent interfaces, and a remainder tabulated from Sommerfeld
 * integrals on 256 log-spaced rho x 128 points in z + z' and in |z - z'|,
 * bilinearly interpolated); the equivalent configuration (Eq. AEFIEeqvdis) uses
 * the homogeneous kernel of layer l.  Plane waves: any incidence from the upper
 * half-space, carried through the stack as TE and TM transmission lines. */
int sldm_stack_create(const sldm_layer* layers, int32_t nlayers, double z_top, int32_t bottom,
                      sldm_stack** out);
int sldm_stack_destroy(sldm_stack* stack);

/* Fill and factor the operator at frequency freq_hz (Sec. II-B to II-E):
 * internal blocks with each object's k, equivalent-configuration blocks with
 * the background's k_l, Y11/Y21 by LU of M_l, global external blocks, I_x.
 * Good conductors (Sec. II-B): a source triangle with an edge longer than
 * 1/|Im k| is bisected through its longest edge, recursively, until no child has
 * an edge longer than 1/|Im k|, and the 6-point rule runs on each child; a fill
 * with split sources drops the pairs whose bounding spheres are more than
 * 40/|Im k| apart.  SLDM_ENOTSUP beyond 4096 children of one source.
 * Objects that repeat an earlier object (same material, same triangles and edges
 * in the same local order, vertices equal up to one translation) take its
 * interior blocks and Y11, Y21; global blocks between object pairs of equal
 * shapes at equal relative placement (and heights, in a stack) are filled once
 * and copied (translation invariance of the kernel).
 * per_obj: nobj materials (host).  The mesh and stack must outlive the op.
 * Errors: SLDM_EINVAL for a non-positive frequency, a material with a
 * non-positive or non-finite eps_r or mu_r or a negative sigma, a current device
 * other than the mesh's, a layer index out of range or an object crossing an
 * interface; SLDM_ENOTSUP for objects in different layers; SLDM_ENOMEM when the
 * device or the budget of sldm_set_device_budget runs out; SLDM_ETIMEOUT when a
 * bounded wait of the batched direct solver runs out.  On every error the call
 * releases what it took and *out is NULL. */
int sldm_assemble(const sldm_mesh* mesh, const sldm_stack* stack, const sldm_material* per_obj,
                  double freq_hz, const sldm_assemble_opts* opts, sldm_op** out);
int sldm_op_info_get(const sldm_op* op, sldm_op_info* info);
/* Copy block `which` (SLDM_BLOCK_*) of object `obj` (ignored for global blocks)
 * into dst as row-major complex128; rows/cols receive its shape.  dst may be
 * NULL to query the shape only. */
int sldm_op_block(const sldm_op* op, int32_t which, int32_t obj, void* dst, int32_t where,
                  int64_t* rows, int64_t* cols);
int sldm_op_destroy(sldm_op* op);
/* Remainder table of a layered operator (verification): which = 0 for the part
 * in (rho, z + z'), 1 for the part in (rho, |z - z'|).  dst receives
 * 5 x nr x n2 complex128 (components xx, phi, zz, z-rho, rho-z; rho log-spaced);
 * dims = {5, nr, n2}; grid = {log rho_min, log rho_max, (z+z')_min, (z+z')_max,
 * |z - z'|_max}.  Host pointers; dst may be NULL.  SLDM_EINVAL if homogeneous. */
int sldm_op_table(const sldm_op* op, int32_t which, void* dst, int64_t* dims, double* grid);

/* y = Z x for nrhs right-hand sides (Eq. finalsystem), column-major N x nrhs
 * complex128 with leading dimension N.  Z is applied in its structured form:
 * global L^A_m, L^phi_m products plus per-object blocks, never a dense Z.
 * SLDM_PREC_F32 operators multiply in FP32; SLDM_PREC_F32X2 operators apply
 * hi + lo with ~48-bit compensated sums (the FP64 operator). */
int sldm_apply(const sldm_op* op, const void* x, void* y, int32_t nrhs, int32_t where, void* stream);

/* Right-hand sides for plane waves (Eq. finalsystem right-hand side):
 * b = [e_inc; 0; 0], e_inc[m] = int f_m . E_inc / eta0,
 * E_inc = pol E0 exp(-j k0 khat . r) with E0 = 1 V/m.
 * khat, pol: nrhs x 3 (real unit direction, real polarisation), host.
 * b: N x nrhs complex128, column-major.  In a stratified background the wave
 * comes from the upper half-space (khat_z < 0, else SLDM_EINVAL) and E_inc is
 * the total field of the stack in the objects' layer: with kt = k0 (khat_x, khat_y),
 * rho = kt / |kt| (at normal incidence the transverse direction of pol) and
 * phi = z x rho, the TE part (E along phi) and the TM part (H along phi) each
 * follow a transmission line in z with line impedances w mu / k_z and
 * k_z / (w eps), continuous transverse E and the reflection coefficient of the
 * layers below at every interface. */
int sldm_rhs_planewave(const sldm_op* op, const double* khat, const double* pol, int32_t nrhs,
                       void* b, int32_t where, void* stream);

/* Solve Z x = b by restarted GMRES with Arnoldi by classical Gram-Schmidt
 * twice and Givens rotations in FP64 (Sec. IV, GMRES); the matrix-vector
 * products, the Krylov basis and the preconditioner's Schur inverses are held
 * in the operator's precision (complex64 operators: FP32 Gram-Schmidt with
 * FP64 sums across threads), right-preconditioned by P of Eq. pcext (Sec. III:
 * diagonals of the blocks, with the analytic block inverse through the Schur
 * complement of the charge block, formed per object at assembly).  Up to 32
 * right-hand sides run in lockstep, each with its own Krylov basis, sharing one
 * multi-RHS pass over the blocks per step (complex64 operators: on the tensor
 * cores from sldm_op_info.tc_from right-hand sides on, else passes of up to 8 on
 * the CUDA cores); more are taken 32 at a time.
 * b, x: N x nrhs complex128 column-major.
 * The iteration runs on the length-scaled system Dr Z Dc (Dr = diag(1, 1, l),
 * Dc = diag(1/l, 1, l) on the blocks [j; e; u], l = the mesh's mean edge
 * length), whose blocks are O(1) for any geometry size in metres; tol and the
 * reported relres refer to ||Dr (b - Z x)|| / ||Dr b||.
 * Complex64 operators (unless refine = SLDM_REFINE_OFF): iterative refinement
 * with an FP64 residual.  The residual at every restart is the product of the
 * stored complex64 blocks with complex128 vectors, accumulated to ~48 bits
 * (exactly split products in compensated FP32 sums), and each
 * GMRES cycle (products in complex64) stops once it has reduced that residual
 * by 1e-5; tol then refers to the FP64 residual of the stored operator.  With
 * SLDM_PREC_F32X2 the residual's operator is hi + lo, the FP64 fill, so tol
 * refers to the FP64 discrete system itself (as with SLDM_PREC_F64).
 * Returns SLDM_ENOTCONV (x holds the last iterate) if tol is not reached. */
int sldm_solve(const sldm_op* op, const void* b, void* x, int32_t nrhs, const sldm_solve_opts* opts,
               sldm_solve_info* info, int32_t where, void* stream);

/* ---- Delta-gap edge ports (Sec. IV-B: a delta-gap edge port at the centre of
 * the dipole, where S11 is measured; Sec. IV-C: two ports on the inductor).
 * A port is the ring of edges of one object lying in the plane s . r = c, each
 * with one triangle on either side; an edge's sign is +1 when its T+ lies on
 * the -s side (the RWG's unit flux crosses the plane along +s).  The source V
 * is an impressed field V delta(s . r - c) s on the surface, entering the
 * external EFIE (row 1 of Eq. finalsystem) as an incident field does:
 * b[edge] = sign V / eta0 on the ring, 0 elsewhere.  The port current is the
 * electric surface current n x H through the ring along +s:
 * I = sum over the ring of sign x[edge] / (j k0) (x[edge] = j k0 H coefficient).
 * Several ports are passed as a CSR on the host: ring_ptr (nports + 1, ring_ptr[0]
 * = 0, every ring non-empty), edges and signs (+1 or -1) of ring p at
 * [ring_ptr[p], ring_ptr[p + 1]).  SLDM_EINVAL for a malformed CSR, an edge out
 * of range or a sign other than +-1. */

/* The ring of object obj in the plane s . r = c (s: 3 doubles, any nonzero
 * length; vertices within tol of the plane, tol <= 0 takes 1e-9 of the mesh's
 * largest extent).  edges, signs: host arrays of capacity cap (may be NULL
 * when cap = 0); *count receives the ring's size, also when it exceeds cap
 * (then SLDM_EINVAL: call again with a larger cap).  SLDM_EINVAL when no edge
 * of the object lies in the plane. */
int sldm_port_ring(const sldm_mesh* m, int32_t obj, const double* s, double c, double tol, int32_t cap,
                   int32_t* edges, int8_t* signs, int32_t* count);

/* Port excitations: column k of b (N x ncols complex128, column-major, `where`)
 * is sum_p V[p + nports k] times port p's right-hand side; V: nports x ncols
 * complex128, column-major, host (V = identity: one port driven per column,
 * the others shorted). */
int sldm_port_rhs(const sldm_op* op, int32_t nports, const int32_t* ring_ptr, const int32_t* edges,
                  const int8_t* signs, const double* V, int32_t ncols, void* b, int32_t where, void* stream);

/* Port currents of solutions x (N x ncols complex128, `where`): I receives
 * nports x ncols complex128, column-major, host.  With the excitations V =
 * identity, I is the admittance matrix Y. */
int sldm_port_currents(const sldm_op* op, int32_t nports, const int32_t* ring_ptr, const int32_t* edges,
                       const int8_t* signs, const void* x, int32_t ncols, double* I, int32_t where, void* stream);

/* Scattering matrix of an n-port from its admittance matrix, for a real
 * reference impedance z0 (ohm) at every port: S = (1 - z0 Y)(1 + z0 Y)^-1, i.e.
 * (Z - z0)(Z + z0)^-1 with Z = Y^-1.  Y, S: n x n complex128, column-major,
 * host.  SLDM_EINVAL for n < 1 or z0 <= 0, SLDM_ENUMERIC when 1 + z0 Y is
 * singular. */
int sldm_port_sparams(int32_t n, const double* Y, double z0, double* S);

/* Bistatic radar cross section (m^2) of the solution x (N complex128, `where`):
 * the equivalent current J_Delta = H - H_eq radiating in the background (Sec.
 * IV-A).  theta, phi, rcs: n doubles, host.  Above a stratified background the
 * observation directions must lie in the upper half-space (0 <= theta < pi/2,
 * else SLDM_EINVAL) and the far field follows by reciprocity: each component is
 * the current's reaction with the stack's plane wave (sldm_rhs_planewave's field)
 * arriving from the observation direction with that polarisation,
 * sigma = eta0^2 (|F_theta|^2 + |F_phi|^2) / (4 pi). */
/* The same for nrhs solutions at once (x: N x nrhs complex128, column-major;
 * rcs: n x nrhs, column-major, host): the phase factors or the stack's waves at
 * each quadrature point are shared by the right-hand sides. */
int sldm_farfield_n(const sldm_op* op, const void* x, int32_t nrhs, int32_t where, const double* theta,
                    const double* phi, int32_t n, double* rcs);
int sldm_farfield(const sldm_op* op, const void* x, int32_t where, const double* theta,
                  const double* phi, int32_t n, double* rcs);

/* Allocation-free Kbar of one object (no counterpart in the paper; it serves
 * callers that cannot allocate device memory).  Some host applications may not
 * call cudaMalloc or cudaFree on their hot path: cudaFree synchronises the whole
 * device and both can stall work that other streams of the process have in
 * flight, and some applications hand all device memory to their own arena under
 * a fixed budget.  This entry point computes the same Kbar(k) of object `obj`
 * as the assembly does (RWG test x BC source, Eq. opKhgf, FP64, without the
 * I_x/2 term of Eq. Kmatdef) into the caller's buffer while allocating nothing:
 * its temporaries live in one file-scope device array of 24 MiB that every GPU
 * which loads the library keeps until the process exits.
 *  - K_out: device pointer, ne_o x ne_o complex128, row-major, written entirely.
 *  - k_re, k_im: complex wavenumber (exp(-j k R) convention, k_im <= 0 decays).
 *  - The object must satisfy ne_o * 9 nt_o <= 1,568,752 (barycentric scratch
 *    entries; about 340 triangles), else SLDM_EINVAL with the sizes in the message.
 *  - Unsplit sources only: when a barycentric triangle has an edge longer than
 *    1/|Im k| (a good conductor, whose assembly splits the sources), SLDM_ENOTSUP.
 *  - Asynchronous on `stream`: K_out is complete when the stream reaches this
 *    point.  Every call shares the one scratch array, which keeps the last call's
 *    contents (the call clears what must start at zero), so calls that overlap
 *    on the GPU (different streams, or different threads) race and must be
 *    serialised by the caller.
 *  - The first call on a device resolves the array's device address with that
 *    device current; make that first call before any stream capture begins.
 *    The address is kept for the life of the process: after cudaDeviceReset (or
 *    anything else that destroys the device's primary context) it is stale, so
 *    do not use this entry point on that device again in the same process. */
int sldm_kbar_noalloc(const sldm_mesh* mesh, int32_t obj, double k_re, double k_im, void* K_out, void* stream);

/* Kernel timers (profiling aid, Sec. IV "CPU time breakdown" counterpart):
 * when enabled, the library records a CUDA event pair around each launch of
 * its main kernels and stages, on the launch's stream, under a fixed name
 * (stages: "assemble", "mgf_tables", "fill_reflected", "apply", "gmres",
 * "gram_schmidt", "precond", "farfield", "nested_y"; kernels: "fill_L_bulk",
 * "fill_L_touch", "fill_L_split", "fill_K_bulk", "fill_K_touch", "fill_K_split",
 * "fill_reflected_bulk", "copy_blocks", "lu_coop", "lu_blocked",
 * "nested_inverse", "gemm_tc" and the product stages "gemv_main", "gemv_y",
 * "gemv_pc", and "gemv_main_f64acc", "gemv_y_f64acc" for the FP64-accurate
 * residual products; names nest, so
 * a stage's time includes its kernels').  Timings are accumulated per name;
 * reading them synchronises on the recorded events.
 * Timed regions pair up within their calling thread, so several threads (the
 * serving workers, each on its own stream) may be timed at once; a region's time
 * then includes whatever else shared the device. */
int sldm_timers_enable(int32_t on);
int sldm_timers_reset(void);
/* Total milliseconds and number of timed launches under `name` (0 if none). */
int sldm_timer_get(const char* name, double* total_ms, int64_t* count);
/* Algorithmic work of the launches timed under `name` since the last reset (the
 * units a roofline divides by the time): "gemv*" the matrix bytes streamed
 * (every entry of every block once per pass, low parts included);
 * "fill_L_bulk", "fill_K_bulk", "fill_reflected_bulk" the Green's-function
 * evaluations (36 per triangle pair the kernel integrates); "gram_schmidt" the
 * Krylov-basis bytes that the two dot and two update passes of classical
 * Gram-Schmidt twice stream.  0 for names without a count. */
int sldm_timer_units(const char* name, double* units);
/* Comma-separated names with recorded launches, NUL-terminated, truncated to len. */
int sldm_timer_names(char* buf, size_t len);
/* Number of kernel launches the library has made in this process (every
 * kernel, timed or not), for counting the launches of a timed region.
 * The paper has no counterpart.  SLDM_EINVAL if out is NULL. */
int sldm_launch_count(int64_t* out);

/* Device-memory budget (the paper has no counterpart; it serves admission
 * control when many operators share one GPU).  The library counts the bytes of
 * every device buffer it holds, over all handles and devices; with a budget of
 * `bytes` > 0 an allocation that would take the count above it fails, and the
 * call that made it returns SLDM_ENOMEM having released what it took.  0 (the
 * default) means no limit.  Buffers already held are not affected by a smaller
 * budget.  SLDM_EINVAL if bytes < 0. */
int sldm_set_device_budget(int64_t bytes);
/* Tensor-core policy of the complex64 products assembled from now on (no
 * counterpart in the paper): 0 (default) measures, per operator, one pass on the
 * tensor cores and as passes of 8 on the CUDA cores at 16 and 32 right-hand sides
 * and sends lockstep widths from the winning point on to the tensor cores
 * (sldm_op_info.tc_from), once per product shape in the process (later operators
 * of the same shape reuse the decision); 1..33 forces that smallest width (33 =
 * never).
 * SLDM_EINVAL otherwise. */
int sldm_set_tc_policy(int32_t tc_from);
/* Bytes of device memory the library holds now (all handles, all devices). */
int sldm_device_bytes(int64_t* in_use);

/* Fault injection for tests of the failure paths (no counterpart in the paper).
 * SLDM_INJECT_LU_STALL: the next `count` launches of the batched direct solver
 * (the cooperative LU of M_l and of the preconditioner's Schur complements) make
 * their first CTA wait first on a device flag that nothing sets.  That wait is
 * bounded like every wait of the solver (a few hundred ms); when it runs out the
 * CTA records the failure, every other CTA leaves at its next wait, and the call
 * that launched the solver (sldm_assemble) returns SLDM_ETIMEOUT.  No fault is
 * raised and the CUDA context stays usable.  count = 0 clears the injection.
 * SLDM_EINVAL for an unknown `what` or a negative count. */
#define SLDM_INJECT_LU_STALL 1
int sldm_test_inject(int32_t what, int32_t count);

/* ---------------------------------------------------------------------------
 * Serving (no counterpart in the paper, which solves one configuration at a
 * time): a request loop over many configurations sharing one GPU.  A request
 * names a registered model (mesh + background + materials), a frequency and
 * plane waves; the server keeps assembled operators resident in a cache keyed by
 * (model, frequency), admits new ones within a device-memory budget by evicting
 * the least recently used operators that no worker is using, solves queued
 * requests of one key together (their right-hand sides in one lockstep GMRES,
 * up to max_batch), and runs `workers` threads, each with its own CUDA stream,
 * so that requests for different operators overlap on the device.  The
 * solution of a request does not depend on what it was batched with beyond the
 * solve tolerance (each right-hand side of a lockstep solve stops on its own
 * residual).
 * ------------------------------------------------------------------------- */
typedef struct sldm_server sldm_server;

typedef struct {
  int32_t workers;      /* worker threads (each with its own CUDA stream), >= 1 */
  int32_t max_batch;    /* right-hand sides per lockstep solve, 1..32 */
  int32_t precision;    /* precision of the cached operators: SLDM_PREC_* */
  int32_t maxit;        /* GMRES iterations per right-hand side (0 = 2000) */
  int64_t budget_bytes; /* device memory for cached operators (0 = no limit) */
} sldm_server_opts;

typedef struct {
  int32_t model;        /* from sldm_server_add_model */
  int32_t nrhs;         /* plane waves, >= 1 (any number: batches split them) */
  double freq_hz;
  const double* khat;   /* nrhs x 3, host; copied by sldm_server_submit */
  const double* pol;    /* nrhs x 3, host; copied by sldm_server_submit */
  double tol;           /* relative residual per right-hand side (0 = 1e-8) */
  void* x;              /* host, N x nrhs complex128 (column-major): receives the
                           solution; borrowed until sldm_server_wait returns */
} sldm_request;

typedef struct {
  int32_t code;         /* SLDM_OK or the failing call's status */
  int32_t iters;        /* GMRES iterations of the solves that carried this request */
  double relres;        /* largest final relative residual of its right-hand sides */
  double t_submit, t_start, t_done; /* seconds on the server's clock */
  int32_t cache_hit;    /* 1 when its operator was resident */
  int32_t batch_rhs;    /* right-hand sides in the lockstep solve that carried it */
} sldm_result;

typedef struct {
  int64_t requests, rhs, batches;      /* completed */
  int64_t hits, misses, evictions, rejected;
  int64_t cached_ops, cached_bytes;    /* now */
  double lat_p50, lat_p99, lat_max;    /* seconds, submit -> done, completed requests */
} sldm_server_stats;

/* Start the workers.  SLDM_EINVAL for invalid options. */
int sldm_server_create(const sldm_server_opts* opts, sldm_server** out);
/* Register a model; the server borrows mesh and stack (they must outlive it) and
 * copies the materials (one per object).  *model receives its id. */
int sldm_server_add_model(sldm_server* srv, const sldm_mesh* mesh, const sldm_stack* stack,
                          const sldm_material* per_obj, int32_t* model);
/* Queue a request; *ticket identifies it for sldm_server_wait.  SLDM_EINVAL for
 * an unknown model or invalid fields. */
int sldm_server_submit(sldm_server* srv, const sldm_request* req, int64_t* ticket);
/* Wait up to timeout_s seconds (< 0: no limit) for a request; fills *res and
 * forgets the ticket.  SLDM_ETIMEOUT if it is still pending (ticket kept),
 * SLDM_EINVAL for an unknown ticket.  The request's own outcome is res->code;
 * when it failed, sldm_last_error in the waiting thread gives the message. */
int sldm_server_wait(sldm_server* srv, int64_t ticket, double timeout_s, sldm_result* res);
int sldm_server_stats_get(sldm_server* srv, sldm_server_stats* st);
/* Drop every cached operator that no worker is using. */
int sldm_server_flush(sldm_server* srv);
/* Finish the queued requests, stop the workers, free the cache. */
int sldm_server_destroy(sldm_server* srv);

/* The server's host-side policies as plain functions (no device work), for
 * checking them without a GPU:
 * sldm_cache_plan: an LRU cache of capacity `budget` bytes (0 = unbounded)
 *   accessed by keys[i] with sizes bytes[i] (same key, same size), i = 0..n-1,
 *   one access at a time and nothing pinned; action[i] = 0 hit, 1 miss admitted,
 *   2 miss larger than the budget (not cached); evicted[i] = entries evicted to
 *   admit access i.
 * sldm_batch_plan: a FIFO queue of n requests (keys[i], nrhs[i]); a batch takes
 *   the oldest request, then the following requests of its key in order while
 *   the right-hand sides fit in max_batch (a request larger than max_batch is a
 *   batch of its own, solved in slices); batch[i] = index of request i's batch,
 *   batches numbered in the order they are formed. */
int sldm_cache_plan(int64_t n, const int64_t* keys, const int64_t* bytes, int64_t budget, int32_t* action,
                    int32_t* evicted);
int sldm_batch_plan(int64_t n, const int64_t* keys, const int32_t* nrhs, int32_t max_batch, int32_t* batch);

#ifdef __cplusplus
}
#endif
#endif /* SLDM_H */
