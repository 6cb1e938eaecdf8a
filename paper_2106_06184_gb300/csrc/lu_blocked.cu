// Blocked right-looking LU with partial pivoting for the large systems of the
// assembly (M_l of an object above ~500 triangles, the preconditioner's Schur
// complement of the same objects): A X = B in place, A n x n and B n x r,
// row-major.  Per panel of NB columns:
//
//   1. lu_panel_kernel   factor the panel [j0, j0 + nb) over rows j0..n-1: one
//                        cooperative launch, every CTA holds a contiguous chunk
//                        of the panel's rows in shared memory; per column a
//                        pivot search across CTAs and an exchange of the pivot
//                        and current rows, two bounded grid barriers;
//   2. lu_swap_kernel    apply the panel's row interchanges to the columns right
//                        of the panel and to B (the L columns left of the panel
//                        are never read again: B is carried along instead);
//   3. lu_trsm_kernel    U12 = L11^-1 A12 (unit lower) on those columns (one
//                        warp per 32 columns, staged in shared memory);
//   4. lu_gemm_kernel    A22 -= L21 U12 on the trailing rows of those columns.
//
// then back substitution U X = B panel by panel from the bottom (upper
// triangular solve on the panel's rows, GEMM update of the rows above).  The
// trailing update carries nearly all the flops; on GB300 the FP64 rate (two
// FMA per SM per clock) is what bounds it, so the tiles are sized for
// occupancy of the FP64 pipe, not for shared-memory reuse.
#include <algorithm>
#include <atomic>

#include "dense.h"

namespace sldm {

namespace {

constexpr int NB = 64;               // panel width
constexpr int PANEL_THREADS = 256;
constexpr int PANEL_MIN_ROWS = 32;   // rows per CTA of the panel factorisation, at least
constexpr unsigned SPIN_LIMIT = 1u << 22;

template <class C>
struct CT2;
template <>
struct CT2<float2> {
  typedef float R;
};
template <>
struct CT2<double2> {
  typedef double R;
};

template <class C>
__device__ __forceinline__ C cmul_(C a, C b) {
  C r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <class C>
__device__ __forceinline__ C cdiv_(C a, C b) {
  typedef typename CT2<C>::R R;
  const R d = b.x * b.x + b.y * b.y;
  C r;
  r.x = (a.x * b.x + a.y * b.y) / d;
  r.y = (a.y * b.x - a.x * b.y) / d;
  return r;
}

// acc += a b and acc -= a b for complex numbers as chains of fused multiply-adds
template <class R>
__device__ __forceinline__ void cfma(R& cr, R& ci, R ar, R ai, R br, R bi) {
  cr = fma(ar, br, cr);
  cr = fma(-ai, bi, cr);
  ci = fma(ar, bi, ci);
  ci = fma(ai, br, ci);
}
template <class R>
__device__ __forceinline__ void cfms(R& cr, R& ci, R ar, R ai, R br, R bi) {
  cr = fma(-ar, br, cr);
  cr = fma(ai, bi, cr);
  ci = fma(-ar, bi, ci);
  ci = fma(-ai, br, ci);
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier over the launch's CTAs (all co-resident: cooperative launch).
// Bounded: a wait that runs out sets *err = 2; every CTA then leaves at its next
// barrier.  Returns false when the kernel must stop (CTA-uniform).
__device__ bool grid_barrier(unsigned* ctr, unsigned target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    int ok = 1;
    unsigned it = 0;
    while (ld_acq(ctr) < target) {
      if (*(volatile int*)err) { ok = 0; break; }
      if (++it > SPIN_LIMIT) { atomicExch(err, 2); ok = 0; break; }
      __nanosleep(32);
    }
    s_ok = ok && !*(volatile int*)err;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- 1. panel
// CTA c holds rows [j0 + c*chunk, min(n, j0 + (c+1)*chunk)) of columns
// [j0, j0 + nb) in shared memory.  Pivot candidates go to slot_v/slot_i[c];
// the pivot row and the current row travel through urow/orow.
template <class C>
__global__ void __launch_bounds__(PANEL_THREADS) lu_panel_kernel(C* A, int n, int j0, int nb, int chunk, int* piv,
                                                                 C* urow, C* orow, double* slot_v, int* slot_i,
                                                                 unsigned* bar, int* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* P = reinterpret_cast<C*>(smem_raw);  // chunk x nb
  C* U = P + size_t(chunk) * nb;          // nb: the current U row
  __shared__ double s_bv[PANEL_THREADS / 32];
  __shared__ int s_bi[PANEL_THREADS / 32];
  __shared__ int s_p;
  const int G = gridDim.x, c = blockIdx.x;
  if (*(volatile int*)err) return;  // an earlier panel failed (uniform across the grid)
  const int r0 = j0 + c * chunk, r1 = min(n, r0 + chunk), nr = max(0, r1 - r0);
  for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    P[t] = A[int64_t(r0 + i) * n + j0 + j];
  }
  __syncthreads();  // the pivot search reads rows loaded by other threads
  unsigned epoch = 0;
  for (int j = 0; j < nb; ++j) {
    const int J = j0 + j;
    // local pivot candidate over rows >= J: largest |a|^2, smallest row on ties
    double best = -1.0;
    int bi = n;
    for (int i = threadIdx.x; i < nr; i += blockDim.x) {
      const int row = r0 + i;
      if (row < J) continue;
      const C a = P[size_t(i) * nb + j];
      const double v = double(a.x) * double(a.x) + double(a.y) * double(a.y);
      if (v > best || (v == best && row < bi)) { best = v; bi = row; }
    }
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { s_bv[threadIdx.x >> 5] = best; s_bi[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < int(blockDim.x >> 5); ++w)
        if (s_bv[w] > s_bv[0] || (s_bv[w] == s_bv[0] && s_bi[w] < s_bi[0])) { s_bv[0] = s_bv[w]; s_bi[0] = s_bi[w]; }
      slot_v[c] = s_bv[0];
      slot_i[c] = s_bi[0];
    }
    if (!grid_barrier(bar, (++epoch) * G, err)) return;
    if (threadIdx.x < 32) {  // warp 0 reduces the G candidates (loads in parallel)
      double b = -1.0;
      int p = n;
      for (int g = threadIdx.x; g < G; g += 32) {
        const double v = __ldcg(slot_v + g);
        const int i = __ldcg(slot_i + g);
        if (v > b || (v == b && i < p)) { b = v; p = i; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, b, o);
        const int oi = __shfl_xor_sync(0xffffffffu, p, o);
        if (ob > b || (ob == b && oi < p)) { b = ob; p = oi; }
      }
      if (threadIdx.x == 0) {
        s_p = (b > 0.0 && p < n) ? p : -1;  // zero, non-finite or missing pivot
        if (s_p < 0 && c == 0) {
          err[1] = J;  // where it stopped
          atomicExch(err, 1);
        }
        if (c == 0 && s_p >= 0) piv[J] = s_p;
      }
    }
    __syncthreads();
    const int p = s_p;
    if (p < 0) return;  // CTA-uniform; the others stop at their next barrier
    // the owners publish the pivot row and the current row
    if (p >= r0 && p < r1)
      for (int t = threadIdx.x; t < nb; t += blockDim.x) urow[t] = P[size_t(p - r0) * nb + t];
    if (J >= r0 && J < r1)
      for (int t = threadIdx.x; t < nb; t += blockDim.x) orow[t] = P[size_t(J - r0) * nb + t];
    if (!grid_barrier(bar, (++epoch) * G, err)) return;
    for (int t = threadIdx.x; t < nb; t += blockDim.x) U[t] = __ldcg(urow + t);
    __syncthreads();
    if (p != J && p >= r0 && p < r1)
      for (int t = threadIdx.x; t < nb; t += blockDim.x) P[size_t(p - r0) * nb + t] = __ldcg(orow + t);
    if (J >= r0 && J < r1)
      for (int t = threadIdx.x; t < nb; t += blockDim.x) P[size_t(J - r0) * nb + t] = U[t];
    __syncthreads();
    // multipliers of the rows below J, then the rank-1 update of the panel's remaining columns
    const C piv_v = U[j];
    for (int i = threadIdx.x; i < nr; i += blockDim.x)
      if (r0 + i > J) P[size_t(i) * nb + j] = cdiv_(P[size_t(i) * nb + j], piv_v);
    __syncthreads();
    const int w = nb - j - 1;
    if (w > 0)
      for (int t = threadIdx.x; t < nr * w; t += blockDim.x) {
        const int i = t / w, cc = 1 + t % w;
        if (r0 + i <= J) continue;
        const C l = P[size_t(i) * nb + j], u = U[j + cc];
        C a = P[size_t(i) * nb + j + cc];
        cfms(a.x, a.y, l.x, l.y, u.x, u.y);
        P[size_t(i) * nb + j + cc] = a;
      }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < nr * nb; t += blockDim.x) {
    const int i = t / nb, j = t % nb;
    A[int64_t(r0 + i) * n + j0 + j] = P[t];
  }
}

// Columns right of the panel: A's columns [ca, n) then B's columns [0, r).
template <class C>
struct Cols {
  C* A;
  int n, ca;
  C* B;
  int r;
  __device__ __forceinline__ int count() const { return (n - ca) + r; }
  // pointer to row 0 of column q of the set, and its row stride
  __device__ __forceinline__ C* col(int q, int64_t& ld) const {
    if (q < n - ca) {
      ld = n;
      return A + ca + q;
    }
    ld = r;
    return B + (q - (n - ca));
  }
};

// ---------------------------------------------------------------- 2. row interchanges
template <class C>
__global__ void lu_swap_kernel(Cols<C> S, int j0, int nb, const int* __restrict__ piv, const int* __restrict__ err) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= S.count() || *err) return;
  int64_t ld = 0;
  C* col = S.col(q, ld);
  for (int j = 0; j < nb; ++j) {
    const int J = j0 + j, p = piv[J];
    if (p != J && p > J && p < S.n) {  // a pivot row is never above its column
      const C a = col[int64_t(J) * ld], b = col[int64_t(p) * ld];
      col[int64_t(J) * ld] = b;
      col[int64_t(p) * ld] = a;
    }
  }
}

// ---------------------------------------------------------------- 3. triangular solves on the panel's rows
// lower = 1: X = L11^-1 X (unit lower, L11 = A[j0.., j0..]); lower = 0: X = U11^-1 X
// (upper, non-unit).  One warp per 32 columns, one thread per column: the nb x nb
// triangle and the warp's nb x 32 block of X are staged in shared memory by
// cp.async (every copy in flight at once), solved there and written back.  The
// FP64 pipe (two FMA per SM per clock) bounds it, so the grid is made of many
// small CTAs to reach every SM.
constexpr int TRSM_COLS = 32;
template <int N>
__device__ __forceinline__ void cp_async_n(void* dst, const void* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if constexpr (N == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
}
template <class C>
__global__ void __launch_bounds__(TRSM_COLS) lu_trsm_kernel(Cols<C> S, const C* __restrict__ A, int n, int j0, int nb,
                                                            int lower, const int* __restrict__ err) {
  if (*err) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* T = reinterpret_cast<C*>(smem_raw);  // nb x nb
  C* X = T + nb * nb;                     // nb x TRSM_COLS
  const int t = threadIdx.x;
  for (int e = t; e < nb * nb; e += TRSM_COLS)
    cp_async_n<sizeof(C)>(T + e, A + int64_t(j0 + e / nb) * n + j0 + e % nb);
  const int q = blockIdx.x * TRSM_COLS + t;
  const bool mine = q < S.count();
  int64_t ld = 0;
  C* col = mine ? S.col(q, ld) + int64_t(j0) * ld : nullptr;
  if (mine)
    for (int k = 0; k < nb; ++k) cp_async_n<sizeof(C)>(X + k * TRSM_COLS + t, col + int64_t(k) * ld);
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  __syncthreads();
  if (!mine) return;
  C* x = X + t;
  if (lower) {
    for (int j = 1; j < nb; ++j) {
      C acc = x[j * TRSM_COLS];
      for (int k = 0; k < j; ++k) {
        const C l = T[j * nb + k], v = x[k * TRSM_COLS];
        cfms(acc.x, acc.y, l.x, l.y, v.x, v.y);
      }
      x[j * TRSM_COLS] = acc;
    }
  } else {
    for (int j = nb - 1; j >= 0; --j) {
      C acc = x[j * TRSM_COLS];
      for (int k = j + 1; k < nb; ++k) {
        const C u = T[j * nb + k], v = x[k * TRSM_COLS];
        cfms(acc.x, acc.y, u.x, u.y, v.x, v.y);
      }
      x[j * TRSM_COLS] = cdiv_(acc, T[j * nb + j]);
    }
  }
  for (int k = 0; k < nb; ++k) col[int64_t(k) * ld] = x[k * TRSM_COLS];
}

// ---------------------------------------------------------------- 4. trailing update
// X[i, q] -= sum_k P[i, k] Q[k, q] for rows i in [i0, i1) of the column set,
// P[i, k] = A[i, kc + k], Q[k, q] = column q of the set at row k0 + k, k < nb.
// 64 x 64 tile per CTA, 256 threads, 4 x 4 results each (columns interleaved).
constexpr int GT = 64;
template <class C>
__global__ void __launch_bounds__(256) lu_gemm_kernel(Cols<C> S, const C* __restrict__ A, int n, int i0, int i1, int kc,
                                                      int k0, int nb, const int* __restrict__ err) {
  if (*err) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Ps = reinterpret_cast<C*>(smem_raw);  // GT x nb
  C* Qs = Ps + GT * nb;                    // nb x GT
  const int rt = i0 + blockIdx.y * GT, qt = blockIdx.x * GT;
  const int nq = S.count();
  for (int t = threadIdx.x; t < GT * nb; t += blockDim.x) {
    const int i = t / nb, k = t % nb;
    C v;
    v.x = 0;
    v.y = 0;
    if (rt + i < i1) v = A[int64_t(rt + i) * n + kc + k];
    Ps[t] = v;
  }
  for (int t = threadIdx.x; t < GT * nb; t += blockDim.x) {
    const int k = t / GT, q = t % GT;
    C v;
    v.x = 0;
    v.y = 0;
    if (qt + q < nq) {
      int64_t ld;
      const C* col = S.col(qt + q, ld);
      v = col[int64_t(k0 + k) * ld];
    }
    Qs[t] = v;
  }
  __syncthreads();
  typedef typename CT2<C>::R R;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  R ar[4][4], ai[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) ar[a][b] = ai[a][b] = R(0);
  for (int k = 0; k < nb; ++k) {
    C p[4], q[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) p[a] = Ps[(ty * 4 + a) * nb + k];
#pragma unroll
    for (int b = 0; b < 4; ++b) q[b] = Qs[k * GT + tx + 16 * b];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        cfma(ar[a][b], ai[a][b], p[a].x, p[a].y, q[b].x, q[b].y);
      }
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int qq = qt + tx + 16 * b;
    if (qq >= nq) continue;
    int64_t ld;
    C* col = S.col(qq, ld);
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = rt + ty * 4 + a;
      if (i >= i1) continue;
      C v = col[int64_t(i) * ld];
      v.x -= ar[a][b];
      v.y -= ai[a][b];
      col[int64_t(i) * ld] = v;
    }
  }
}

}  // namespace

template <class C>
void lu_solve_blocked(const LUSysT<C>& S, cudaStream_t s) {
  const int n = S.n, r = S.nrhs;
  int dev = 0, nsm = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  SLDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  DBuf<int> piv, err;
  DBuf<C> urow, orow;
  DBuf<double> slot_v;
  DBuf<int> slot_i;
  DBuf<unsigned> bar;
  piv.alloc(n);
  SLDM_CUDA(cudaMemsetAsync(piv.p, 0xff, size_t(n) * sizeof(int), s));  // -1: no pivot yet
  err.alloc(2);
  err.zero(s);
  urow.alloc(NB);
  orow.alloc(NB);
  slot_v.alloc(nsm);
  slot_i.alloc(nsm);
  bar.alloc(1);
  const int max_chunk = (n + nsm - 1) / nsm > PANEL_MIN_ROWS ? (n + nsm - 1) / nsm : PANEL_MIN_ROWS;
  const size_t panel_smem = (size_t(max_chunk) * NB + NB) * sizeof(C);
  SLDM_REQUIRE(panel_smem <= 200 * 1024, SLDM_ENOTSUP, "LU: panel too large for shared memory");
  {
    // per function and context, shared by every launching thread: set once to the
    // largest size accepted above, never to this call's size
    static std::atomic<uint64_t> set{0};
    int dev = 0;
    SLDM_CUDA(cudaGetDevice(&dev));
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(set.load() & bit)) {
      SLDM_CUDA(cudaFuncSetAttribute(lu_panel_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
      set.fetch_or(bit);
    }
  }
  int per_sm = 0;
  SLDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_panel_kernel<C>, PANEL_THREADS, panel_smem));
  SLDM_REQUIRE(per_sm >= 1, SLDM_ENOTSUP, "LU: panel kernel does not fit on an SM");
  const size_t trsm_smem = (size_t(NB) * NB + size_t(NB) * TRSM_COLS) * sizeof(C);
  const size_t gemm_smem = size_t(2) * GT * NB * sizeof(C);
  SLDM_CUDA(cudaFuncSetAttribute(lu_trsm_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(trsm_smem)));
  SLDM_CUDA(cudaFuncSetAttribute(lu_gemm_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(gemm_smem)));
  ScopedTimer tm("lu_blocked", s);
  for (int j0 = 0; j0 < n; j0 += NB) {
    const int nb = std::min(NB, n - j0);
    const int rows = n - j0;
    const int G = std::max(1, std::min(nsm, (rows + PANEL_MIN_ROWS - 1) / PANEL_MIN_ROWS));
    const int chunk = (rows + G - 1) / G;
    SLDM_CUDA(cudaMemsetAsync(bar.p, 0, sizeof(unsigned), s));
    {
      C* a0 = S.A;
      int a1 = n, a2 = j0, a3 = nb, a4 = chunk;
      int* a5 = piv.p;
      C* a6 = urow.p;
      C* a7 = orow.p;
      double* a8 = slot_v.p;
      int* a9 = slot_i.p;
      unsigned* a10 = bar.p;
      int* a11 = err.p;
      void* args[] = {&a0, &a1, &a2, &a3, &a4, &a5, &a6, &a7, &a8, &a9, &a10, &a11};
      const size_t sm = (size_t(chunk) * NB + NB) * sizeof(C);
      SLDM_CUDA(cudaLaunchCooperativeKernel((void*)lu_panel_kernel<C>, dim3(G), dim3(PANEL_THREADS), args, sm, s));
      count_launch();
    }
    Cols<C> R{S.A, n, j0 + nb, S.B, r};
    const int nq = (n - j0 - nb) + r;
    if (nq > 0) {
      lu_swap_kernel<C><<<(nq + 255) / 256, 256, 0, s>>>(R, j0, nb, piv.p, err.p), count_launch();
      lu_trsm_kernel<C><<<(nq + TRSM_COLS - 1) / TRSM_COLS, TRSM_COLS, trsm_smem, s>>>(R, S.A, n, j0, nb, 1, err.p),
          count_launch();
      if (j0 + nb < n) {
        dim3 grid((nq + GT - 1) / GT, (n - j0 - nb + GT - 1) / GT);
        lu_gemm_kernel<C><<<grid, 256, gemm_smem, s>>>(R, S.A, n, j0 + nb, n, j0, j0, nb, err.p), count_launch();
      }
    }
    SLDM_CUDA(cudaGetLastError());
  }
  // back substitution U X = B on B's columns, panels from the bottom
  if (r > 0) {
    Cols<C> Bc{S.A, n, n, S.B, r};
    const int npan = (n + NB - 1) / NB;
    for (int p = npan - 1; p >= 0; --p) {
      const int j0 = p * NB, nb = std::min(NB, n - j0);
      lu_trsm_kernel<C><<<(r + TRSM_COLS - 1) / TRSM_COLS, TRSM_COLS, trsm_smem, s>>>(Bc, S.A, n, j0, nb, 0, err.p),
          count_launch();
      if (j0 > 0) {
        dim3 grid((r + GT - 1) / GT, (j0 + GT - 1) / GT);
        lu_gemm_kernel<C><<<grid, 256, gemm_smem, s>>>(Bc, S.A, n, 0, j0, j0, j0, nb, err.p), count_launch();
      }
    }
    SLDM_CUDA(cudaGetLastError());
  }
  int herr[2] = {0, 0};
  SLDM_CUDA(cudaMemcpyAsync(herr, err.p, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  SLDM_REQUIRE(herr[0] != 2, SLDM_ETIMEOUT, "LU: a panel barrier ran out of its wait limit");
  SLDM_REQUIRE(herr[0] == 0, SLDM_ENUMERIC,
               "LU: zero or non-finite pivot in column " + std::to_string(herr[1]) + " of " + std::to_string(n));
}

template void lu_solve_blocked<float2>(const LUSysT<float2>&, cudaStream_t);
template void lu_solve_blocked<double2>(const LUSysT<double2>&, cudaStream_t);

}  // namespace sldm
