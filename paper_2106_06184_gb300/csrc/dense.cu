// Dense algebra of the SLDM system on the device:
//  - M_l and its right-hand side [Kbar_l + I_x/2; 0] per object (Eq. AEFIEeqvdis),
//    batched LU with partial pivoting in FP64 -> Y11, Y21 (Eq. Yeqdef);
//  - batched skinny GEMV (y = alpha A x + beta y, up to 8 right-hand sides per
//    pass) streaming row-major complex blocks once per pass: the HBM-bound
//    matrix-vector product that drives GMRES;
//  - the sparse/elementwise glue of the structured product Z x (Eq. finalsystem);
//  - vector kernels for GMRES (Arnoldi by classical Gram-Schmidt twice), in the
//    Krylov basis' precision, batched over the lockstep right-hand sides.
#include <algorithm>
#include <atomic>
#include <tuple>
#include <mutex>
#include <map>
#include <type_traits>

#include "dense.h"
#include "gemm_tc.h"

namespace sldm {

template <class C>
struct CT;
template <>
struct CT<float2> {
  typedef float R;
};
template <>
struct CT<double2> {
  typedef double R;
};

// acc += a b and acc -= a b for complex numbers as chains of fused multiply-adds:
// four per complex product (a sum of two products written as one expression
// compiles to a multiply, an FMA and an add, and the FP64 pipe is the bound).
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

// ---------------------------------------------------------------- M_l and R_l
// M_l is built length-scaled (l = mean edge length): Mh = diag(1, l) M_l diag(1/l, l)
// = [[mu_l L^A_l / l, -l D^T L^phi_l B], [F D, -k0^2 l^2 I]], whose entries are O(1);
// its solution Yh gives Y11 = Yh11 / l and Y21 = l Yh21 (the right-hand side is unchanged).
template <class C>
__global__ void build_Ml_kernel(int ne_o, int nt_o, int e0, int t0, double k0, double ell, const C* __restrict__ LAm, int64_t ldLA,
                                const C* __restrict__ LPm, int64_t ldLP, const int32_t* __restrict__ tplus,
                                const int32_t* __restrict__ tminus, C* Ml) {
  const int n = ne_o + nt_o - 1;
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (col >= n) return;
  double2 v = make_double2(0, 0);
  if (row < ne_o && col < ne_o) {
    C a = LAm[int64_t(e0 + row) * ldLA + (e0 + col)];
    v = make_double2(double(a.x) / ell, double(a.y) / ell);
  } else if (row < ne_o) {
    // -(D^T L^phi_m B)[row, q]:  (L B)[t, q] = L[t, q] - L[t, last]
    int q = col - ne_o;
    int last = t0 + nt_o - 1;
    int tp = tplus[e0 + row], tm = tminus[e0 + row];
    C a = LPm[int64_t(tp) * ldLP + (t0 + q)], b = LPm[int64_t(tp) * ldLP + last];
    C c = LPm[int64_t(tm) * ldLP + (t0 + q)], d = LPm[int64_t(tm) * ldLP + last];
    double re = (double(a.x) - double(b.x)) - (double(c.x) - double(d.x));
    double im = (double(a.y) - double(b.y)) - (double(c.y) - double(d.y));
    v = make_double2(-re * ell, -im * ell);
  } else if (col < ne_o) {
    // (F D)[q, col]: +1 if triangle q is T+ of edge col, -1 if T-
    int q = row - ne_o;
    int tp = tplus[e0 + col] - t0, tm = tminus[e0 + col] - t0;
    v = make_double2((tp == q ? 1.0 : 0.0) - (tm == q ? 1.0 : 0.0), 0.0);
  } else {
    v = make_double2(row == col ? -k0 * k0 * ell * ell : 0.0, 0.0);
  }
  C o;
  o.x = decltype(o.x)(v.x);
  o.y = decltype(o.y)(v.y);
  Ml[int64_t(row) * n + col] = o;
}

// R = [Kbar_l + I_x/2 ; 0]  (n x ne_o, row-major)
template <class C>
__global__ void build_Rl_kernel(int ne_o, int nt_o, int e0, const C* __restrict__ Kl, int64_t ldK,
                                const int32_t* __restrict__ ix_ptr, const int32_t* __restrict__ ix_col,
                                const double* __restrict__ ix_val, C* Rl) {
  int col = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (col >= ne_o) return;
  double2 v = make_double2(0, 0);
  if (row < ne_o) {
    C a = Kl[int64_t(row) * ldK + col];
    v = make_double2(double(a.x), double(a.y));
    for (int z = ix_ptr[e0 + row]; z < ix_ptr[e0 + row + 1]; ++z)
      if (ix_col[z] == e0 + col) v.x += 0.5 * ix_val[z];
  }
  C o;
  o.x = decltype(o.x)(v.x);
  o.y = decltype(o.y)(v.y);
  Rl[int64_t(row) * ne_o + col] = o;
}

template <class C>
void build_Ml(const sldm_mesh* m, int obj, double k0, const void* LAm, int64_t ldLA, const void* LPm, int64_t ldLP,
              const void* Kl, int64_t ldK, const double* ix_val, C* Ml, C* Rl, cudaStream_t s) {
  const HostMesh& h = m->h;
  int e0 = h.edge_begin[obj], ne_o = h.edge_begin[obj + 1] - e0;
  int t0 = h.tri_begin[obj], nt_o = h.tri_begin[obj + 1] - t0;
  int n = ne_o + nt_o - 1;
  build_Ml_kernel<C><<<dim3((n + 127) / 128, n), 128, 0, s>>>(ne_o, nt_o, e0, t0, k0, h.ell, (const C*)LAm, ldLA, (const C*)LPm,
                                                              ldLP, m->d.tplus.p, m->d.tminus.p, Ml), ::sldm::count_launch();
  build_Rl_kernel<C><<<dim3((ne_o + 127) / 128, n), 128, 0, s>>>(ne_o, nt_o, e0, (const C*)Kl, ldK, m->d.ix_ptr.p,
                                                                 m->d.ix_col.p, ix_val, Rl), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- batched LU (FP64)
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// Batched LU with partial pivoting and look-ahead, one cooperative launch.
// The CTAs are split into groups, one group per system (or one CTA per system
// when there are more systems than CTAs).  Within a group the columns of
// [A | B] are owned block-cyclically (blocks of two columns) by the group's
// CTAs.  Column k is "published" by its owner: pivot row p_k in piv_row[k],
// pivot in diag[k], the multipliers of rows > k (of the row-swapped column) in
// place, then flag[k] = 1.  At step k every CTA waits for flag[k], swaps rows
// k and p_k of its own columns and eliminates their rows > k; the owner of
// column k+1 does that column first and publishes it before touching the rest,
// so no step needs a barrier across the group.  The right-hand sides are
// eliminated in the same sweep; after one group barrier each CTA
// back-substitutes the right-hand-side columns it owns.
//
// Every wait is bounded: a wait that runs out records an error, after which
// every CTA leaves at its next wait.
constexpr int LU_THREADS = 512;
constexpr unsigned LU_SPIN_LIMIT = 1u << 22;

struct LUGroup {
  int32_t sys0, nsys_stride;  // systems handled: sys0, sys0 + stride, ... (< nsys)
  int32_t cta0, gs;           // first CTA and size of the group
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" : : "l"(p), "r"(v) : "memory");
}

// Thread 0 waits until *p >= target (bounded), then the CTA continues.
// Returns false when the kernel must stop.
__device__ bool wait_at_least(const unsigned* p, unsigned target, int* err) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned it = 0;
    while (ld_acquire(p) < target) {
      if (*(volatile int*)err) { ok = 0; break; }
      if (++it > LU_SPIN_LIMIT) { atomicExch(err, 2); ok = 0; break; }
      __nanosleep(32);
    }
    s_ok = ok && !*(volatile int*)err;
  }
  __syncthreads();
  return s_ok != 0;
}

template <class C>
__device__ __forceinline__ C* lu_colptr(const LUSysT<C>& S, int J) { return J < S.n ? S.A + J : S.B + (J - S.n); }
__device__ __forceinline__ int lu_owner(int J, int gs) { return (J >> 1) % gs; }

// Pivot search over v[0..m) (rows base..base+m-1): largest |v|^2, smallest row on ties.
template <class C>
__device__ void lu_argmax(const C* v, int m, int base, int* out_p) {
  __shared__ double s_bv[LU_THREADS / 32];
  __shared__ int s_bi[LU_THREADS / 32];
  double best = -1.0;
  int bi = base;
  for (int t = threadIdx.x; t < m; t += blockDim.x) {
    const double a = double(v[t].x) * double(v[t].x) + double(v[t].y) * double(v[t].y);
    if (a > best || (a == best && base + t < bi)) { best = a; bi = base + t; }
  }
  for (int o = 16; o > 0; o >>= 1) {
    double ob = __shfl_xor_sync(0xffffffffu, best, o);
    int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if ((threadIdx.x & 31) == 0) { s_bv[threadIdx.x >> 5] = best; s_bi[threadIdx.x >> 5] = bi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = s_bv[0];
    int p = s_bi[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
      if (s_bv[w] > b || (s_bv[w] == b && s_bi[w] < p)) { b = s_bv[w]; p = s_bi[w]; }
    *out_p = (b > 0.0) ? p : -1;
  }
  __syncthreads();
}

// Publishes column J (its rows J.. already hold the values of all earlier
// steps, copied to v[0..n-J)): pivot, row swap, multipliers, flag.
template <class C>
__device__ void lu_publish(const LUSysT<C>& S, int J, C* v, C* diag, int* piv_row, unsigned* flag, int* err) {
  typedef decltype(v->x) R;
  __shared__ int s_p;
  const int n = S.n, m = n - J;
  lu_argmax(v, m, J, &s_p);
  const int p = s_p;
  if (p < 0) {
    if (threadIdx.x == 0) atomicExch(err, 1);  // zero or non-finite pivot
    __syncthreads();
    return;
  }
  const C piv = v[p - J];
  const R den = piv.x * piv.x + piv.y * piv.y;
  C* col = S.A + J;
  for (int t = 1 + threadIdx.x; t < m; t += blockDim.x) {
    const int i = J + t;
    const C a = (i == p) ? v[0] : v[t];
    C q;
    q.x = (a.x * piv.x + a.y * piv.y) / den;
    q.y = (a.y * piv.x - a.x * piv.y) / den;
    col[int64_t(i) * n] = q;
  }
  if (threadIdx.x == 0) {
    col[int64_t(J) * n] = piv;
    diag[J] = piv;
    piv_row[J] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flag + J, 1u);
  }
}

template <class C>
__global__ void __launch_bounds__(LU_THREADS) lu_coop_kernel(const LUSysT<C>* __restrict__ sys, int nsys,
                                                             const LUGroup* __restrict__ groups, const int* __restrict__ cta_group,
                                                             C* diag_all, int* pivrow_all, unsigned* flag_all,
                                                             const int64_t* __restrict__ off, unsigned* ctr, int* err,
                                                             int max_own, const unsigned* stall_flag) {
  typedef decltype(diag_all->x) R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* smem = reinterpret_cast<C*>(smem_raw);
  // injected failure (sldm_test_inject): CTA 0 first waits on a flag that nothing
  // sets; the wait runs out, records err = 2 and every CTA leaves at its next wait
  if (stall_flag != nullptr && blockIdx.x == 0 && !wait_at_least(stall_flag, 1u, err)) return;
  const int gid = cta_group[blockIdx.x];
  const LUGroup G = groups[gid];
  const int rank = blockIdx.x - G.cta0;
  unsigned epoch = 0;
  for (int si = G.sys0; si < nsys; si += G.nsys_stride) {
    __syncthreads();
    const LUSysT<C> S = sys[si];
    const int n = S.n, r = S.nrhs, ncol = n + r;
    C* diag = diag_all + off[si];
    int* piv_row = pivrow_all + off[si];
    unsigned* flag = flag_all + off[si];
    C* colv = smem;            // n: working copy of the column being published
    C* mult = colv + n;        // n: multipliers of the current step
    C* rowk = mult + n;        // max_own
    C* rowp = rowk + max_own;  // max_own
    int* own = reinterpret_cast<int*>(rowp + max_own);
    int nown = 0;
    for (int b = rank; 2 * b < ncol; b += G.gs)
      for (int jj = 0; jj < 2; ++jj)
        if (2 * b + jj < ncol) {
          if (threadIdx.x == 0) own[nown] = 2 * b + jj;
          ++nown;
        }
    __syncthreads();
    // column 0 is published by its owner before the first step
    if (lu_owner(0, G.gs) == rank) {
      for (int t = threadIdx.x; t < n; t += blockDim.x) colv[t] = S.A[int64_t(t) * n];
      __syncthreads();
      lu_publish(S, 0, colv, diag, piv_row, flag, err);
    }
    int first = 0;
    for (int k = 0; k < n; ++k) {
      if (!wait_at_least(flag + k, 1u, err)) return;
      while (first < nown && own[first] <= k) ++first;
      const int p = __ldcg(piv_row + k);
      const int rows = n - k - 1;
      const int na = nown - first;
      for (int t = threadIdx.x; t < rows; t += blockDim.x) mult[t] = __ldcg(S.A + int64_t(k + 1 + t) * n + k);
      for (int c = threadIdx.x; c < na; c += blockDim.x) {
        const int J = own[first + c];
        const C* col = lu_colptr(S, J);
        const int64_t ld = J < n ? n : r;
        rowk[c] = __ldcg(col + int64_t(k) * ld);
        rowp[c] = __ldcg(col + int64_t(p) * ld);
      }
      __syncthreads();
      // look-ahead: the owner of column k+1 eliminates and publishes it first
      int skip = -1;
      if (k + 1 < n && lu_owner(k + 1, G.gs) == rank) {
        const int c = 0;  // own[first] == k + 1 for the owner of column k + 1
        skip = c;
        C* col = S.A + (k + 1);
        const C u = rowp[c];
        for (int t = threadIdx.x; t <= rows; t += blockDim.x) {
          // t = 0 is row k (takes row p), t >= 1 are rows k + t
          if (t == 0) continue;
          const int i = k + t;
          const C l = mult[t - 1];
          C a = (i == p) ? rowk[c] : __ldcg(col + int64_t(i) * n);
          cfms(a.x, a.y, l.x, l.y, u.x, u.y);
          colv[t - 1] = a;  // rows k+1 .. n-1
        }
        if (threadIdx.x == 0) col[int64_t(k) * n] = u;
        __syncthreads();
        lu_publish(S, k + 1, colv, diag, piv_row, flag, err);
      }
      // the other owned columns
      const int c0 = (skip == 0) ? 1 : 0;
      const int nb = na - c0;
      if (p != k)
        for (int c = c0 + threadIdx.x; c < na; c += blockDim.x) {
          const int J = own[first + c];
          C* col = lu_colptr(S, J);
          col[int64_t(k) * (J < n ? n : r)] = rowp[c];
        }
      const int64_t work = int64_t(rows) * nb;
      for (int64_t w0 = threadIdx.x; w0 < work; w0 += 4 * int64_t(blockDim.x)) {
        C a[4];
        int64_t addr[4];
        C* base[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t w = w0 + int64_t(q) * blockDim.x;
          base[q] = nullptr;
          if (w < work) {
            const int t = int(w / nb), c = c0 + int(w % nb);
            const int i = k + 1 + t;
            const int J = own[first + c];
            base[q] = lu_colptr(S, J);
            addr[q] = int64_t(i) * (J < n ? n : r);
            a[q] = (i == p) ? rowk[c] : __ldcg(base[q] + addr[q]);
          }
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t w = w0 + int64_t(q) * blockDim.x;
          if (w < work) {
            const int t = int(w / nb), c = c0 + int(w % nb);
            const C l = mult[t];
            const C u = rowp[c];
            C v = a[q];
            cfms(v.x, v.y, l.x, l.y, u.x, u.y);
            base[q][addr[q]] = v;
          }
        }
      }
      __syncthreads();
      // errors are acted on at the next (CTA-uniform) wait
    }
    // every column is final once every CTA of the group has finished its last step
    ++epoch;
    if (G.gs > 1) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr + gid, 1u);
      }
      if (!wait_at_least(ctr + gid, epoch * G.gs, err)) return;
    }
    // ---- back substitution U X = B on the owned right-hand-side columns
    int rfirst = 0;
    while (rfirst < nown && own[rfirst] < n) ++rfirst;
    const int nr = nown - rfirst;
    C* ys = rowk;
    for (int k = n - 1; k >= 0 && nr > 0; --k) {
      const C dk = __ldcg(diag + k);
      const R dd = dk.x * dk.x + dk.y * dk.y;
      for (int c = threadIdx.x; c < nr; c += blockDim.x) {
        C* col = S.B + (own[rfirst + c] - n);
        const C bk = __ldcg(col + int64_t(k) * r);
        C y;
        y.x = (bk.x * dk.x + bk.y * dk.y) / dd;
        y.y = (bk.y * dk.x - bk.x * dk.y) / dd;
        ys[c] = y;
        col[int64_t(k) * r] = y;
      }
      __syncthreads();
      const int64_t work = int64_t(k) * nr;
      for (int64_t w = threadIdx.x; w < work; w += blockDim.x) {
        const int i = int(w / nr), c = int(w % nr);
        C* col = S.B + (own[rfirst + c] - n);
        const C u = __ldcg(S.A + int64_t(i) * n + k);
        const C y = ys[c];
        C v = __ldcg(col + int64_t(i) * r);
        cfms(v.x, v.y, u.x, u.y, y.x, y.y);
        col[int64_t(i) * r] = v;
      }
      __syncthreads();
    }
    // the next system of this group starts only after every CTA finished this one
    ++epoch;
    if (G.gs > 1) {
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(ctr + gid, 1u);
      }
      if (!wait_at_least(ctr + gid, epoch * G.gs, err)) return;
    }
  }
}

template <class C>
void lu_solve_batched(const std::vector<LUSysT<C>>& all, cudaStream_t s) {
  std::vector<LUSysT<C>> systems;
  for (auto& S : all) {
    if (S.n >= LU_BLOCKED_MIN) lu_solve_blocked<C>(S, s);
    else systems.push_back(S);
  }
  if (systems.empty()) return;
  int dev = 0, nsm = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  SLDM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  int coop = 0;
  SLDM_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  SLDM_REQUIRE(coop, SLDM_ENOTSUP, "LU: device does not support cooperative launches");
  int nmax = 0, cmax = 0;
  for (auto& S : systems) {
    nmax = std::max(nmax, S.n);
    cmax = std::max(cmax, S.n + S.nrhs);
  }
  const int nsys_ = int(systems.size());
  const int gs_min = nsys_ <= nsm ? nsm / nsys_ : 1;
  const int max_own = 2 * ((cmax + 1) / 2 / gs_min + 1);
  const size_t smem = size_t(2) * nmax * sizeof(C) + size_t(2) * max_own * sizeof(C) + size_t(max_own) * sizeof(int);
  SLDM_REQUIRE(smem <= 220 * 1024, SLDM_ENOTSUP,
               "LU: object too large for the in-kernel direct factorisation (n = " + std::to_string(nmax) + ")");
  {
    // the limit is per function and context, shared by every thread that launches
    // it: set once to the largest size accepted above, never to this call's size
    static std::atomic<uint64_t> set{0};
    const uint64_t bit = uint64_t(1) << (dev & 63);
    if (!(set.load() & bit)) {
      SLDM_CUDA(cudaFuncSetAttribute(lu_coop_kernel<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
      set.fetch_or(bit);
    }
  }
  int per_sm = 0;
  SLDM_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, lu_coop_kernel<C>, LU_THREADS, smem));
  SLDM_REQUIRE(per_sm >= 1, SLDM_ENOTSUP, "LU: kernel does not fit on an SM");
  const int nsys = int(systems.size());
  const int G = nsm;  // one CTA per SM
  std::vector<LUGroup> groups;
  std::vector<int> cta_group(G);
  if (nsys <= G) {
    const int gs = G / nsys;
    for (int g = 0; g < nsys; ++g) groups.push_back({g, nsys, g * gs, gs});
    for (int b = 0; b < G; ++b) cta_group[b] = std::min(b / gs, nsys - 1);
    // CTAs beyond nsys * gs join the last group's range but own no columns: extend the last group
    groups.back().gs = G - groups.back().cta0;
  } else {
    for (int g = 0; g < G; ++g) groups.push_back({g, G, g, 1});
    for (int b = 0; b < G; ++b) cta_group[b] = b;
  }
  std::vector<int64_t> doff(nsys);
  int64_t dtot = 0;
  for (int i = 0; i < nsys; ++i) {
    doff[i] = dtot;
    dtot += systems[i].n;
  }
  DBuf<LUSysT<C>> d;
  DBuf<LUGroup> dg;
  DBuf<int> dcg, err;
  DBuf<int64_t> ddo;
  DBuf<C> diag;
  DBuf<int> pivrow;
  DBuf<unsigned> ctr, flags;
  d.upload(systems, s);
  dg.upload(groups, s);
  dcg.upload(cta_group, s);
  ddo.upload(doff, s);
  diag.alloc(dtot);
  pivrow.alloc(dtot);
  flags.alloc(dtot);
  flags.zero(s);
  ctr.alloc(groups.size() + 1);  // one more: the flag of an injected stall, never set
  ctr.zero(s);
  err.alloc(1);
  err.zero(s);
  const LUSysT<C>* a0 = d.p;
  int a1 = nsys;
  const LUGroup* a2 = dg.p;
  const int* a3 = dcg.p;
  C* a4 = diag.p;
  int* a5 = pivrow.p;
  unsigned* a6 = flags.p;
  const int64_t* a7 = ddo.p;
  unsigned* a8 = ctr.p;
  int* a9 = err.p;
  int a10 = max_own;
  const unsigned* a11 = take_lu_stall() ? ctr.p + groups.size() : nullptr;
  void* args[] = {(void*)&a0, (void*)&a1, (void*)&a2, (void*)&a3, (void*)&a4, (void*)&a5,
                  (void*)&a6, (void*)&a7, (void*)&a8, (void*)&a9, (void*)&a10, (void*)&a11};
  {
    ScopedTimer tm("lu_coop", s);
    SLDM_CUDA(cudaLaunchCooperativeKernel((void*)lu_coop_kernel<C>, dim3(G), dim3(LU_THREADS), args, smem, s));
    count_launch();
  }
  int herr = 0;
  SLDM_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  SLDM_CUDA(cudaStreamSynchronize(s));
  SLDM_REQUIRE(herr != 2, SLDM_ETIMEOUT, "LU: a wait for a published column ran out of its limit");
  SLDM_REQUIRE(herr == 0, SLDM_ENUMERIC, "LU of M_l: zero or non-finite pivot");
}
template void lu_solve_batched<float2>(const std::vector<LUSysT<float2>>&, cudaStream_t);
template void lu_solve_batched<double2>(const std::vector<LUSysT<double2>>&, cudaStream_t);

// ---------------------------------------------------------------- batched skinny GEMV
// One right-hand side (instantiated with NR = 1; several go to the row-tile
// kernel below).  Each warp owns one row of one job; rows are split over jobs
// by an exclusive prefix sum.  The matrix entries are CM (complex64 or
// complex128) and stream through once with two 16-byte loads per lane in
// flight; the vectors and the accumulation are CV.
template <class CM, class CV, int NR>
__global__ void __launch_bounds__(256, NR == 1 ? 6 : 1) gemv_jobs_kernel(const GemvJob* __restrict__ jobs, const int64_t* __restrict__ rowstart,
                                                        int njobs, int64_t total_rows, int nrhs) {
  typedef typename CT<CV>::R R;
  const int64_t warp = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= total_rows) return;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (rowstart[mid] <= warp) lo = mid;
    else hi = mid - 1;
  }
  const GemvJob J = jobs[lo];
  const int64_t row = warp - rowstart[lo];
  const CM* __restrict__ A = reinterpret_cast<const CM*>(J.A) + row * J.lda;
  const CV* __restrict__ x = reinterpret_cast<const CV*>(J.x);
  R accr[NR], acci[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) accr[r] = acci[r] = R(0);
  auto mac1 = [&](const CM a, int c) {
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) {
        const CV xv = x[int64_t(r) * J.ldx + c];
        cfma(accr[r], acci[r], R(a.x), R(a.y), R(xv.x), R(xv.y));
      }
  };
  int c0 = 0;  // first column left to the scalar loop
  if (sizeof(CM) == 8 && ((reinterpret_cast<uintptr_t>(A) & 15) == 0)) {
    // complex64: 16-byte loads of two consecutive entries
    const int n2 = J.n / 2;
    const float4* A4 = reinterpret_cast<const float4*>(A);
    auto mac2 = [&](const float4 a, int c) {
#pragma unroll
      for (int r = 0; r < NR; ++r)
        if (r < nrhs) {
          const CV x0 = x[int64_t(r) * J.ldx + 2 * c], x1 = x[int64_t(r) * J.ldx + 2 * c + 1];
          cfma(accr[r], acci[r], R(a.x), R(a.y), R(x0.x), R(x0.y));
          cfma(accr[r], acci[r], R(a.z), R(a.w), R(x1.x), R(x1.y));
        }
    };
    int c = lane;
    for (; c + 32 < n2; c += 64) {
      const float4 a0 = __ldcs(A4 + c), a1 = __ldcs(A4 + c + 32);
      mac2(a0, c);
      mac2(a1, c + 32);
    }
    if (c < n2) mac2(__ldcs(A4 + c), c);
    c0 = 2 * n2;
  } else if (sizeof(CM) == 16) {
    int c = lane;
    for (; c + 32 < J.n; c += 64) {
      const CM a0 = __ldcs(A + c), a1 = __ldcs(A + c + 32);
      mac1(a0, c);
      mac1(a1, c + 32);
    }
    if (c < J.n) mac1(__ldcs(A + c), c);
    c0 = J.n;
  }
  for (int c = c0 + lane; c < J.n; c += 32) mac1(A[c], c);
#pragma unroll
  for (int r = 0; r < NR; ++r) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      accr[r] += __shfl_xor_sync(0xffffffffu, accr[r], o);
      acci[r] += __shfl_xor_sync(0xffffffffu, acci[r], o);
    }
  }
  if (lane == 0) {
    CV* y = reinterpret_cast<CV*>(J.y);
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) {
        R vr = R(J.ar) * accr[r] - R(J.ai) * acci[r];
        R vi = R(J.ar) * acci[r] + R(J.ai) * accr[r];
        CV* yy = y + int64_t(r) * J.ldy + row;
        if (J.beta) {
          vr += yy->x;
          vi += yy->y;
        }
        yy->x = vr;
        yy->y = vi;
      }
  }
}

// ---------------------------------------------------------------- several right-hand sides
// With NR right-hand sides every matrix entry feeds 4 NR FMAs, so at NR = 8 a
// complex64 pass needs 32 FP32 FMAs per 8 bytes streamed: the one-row-per-warp
// kernel above, which re-reads x from L1 for every row, is load-issue bound
// there.  This kernel gives each warp RW rows and each CTA 8 RW consecutive
// rows of one job, stages x once per CTA in shared memory and streams A
// through a 4-stage cp.async pipeline (each lane copies, then reads back, its
// own entries; the x chunk is shared, so a CTA barrier guards each stage).
// Columns go in chunks of 64, two per lane; entries outside the block or
// beyond nrhs are zero-filled by the copy, so the inner loop has no branches.
// The partial sums are reduced by a transposing butterfly that halves the
// values held per lane at every step (about 2K shuffles for K values rather
// than 5K) and leaves each lane with the sums it writes.
template <class CM, class CV>
struct GemvTile {
  static constexpr int RW = sizeof(CV) == 8 ? 4 : 2;  // rows per warp
  static constexpr int CW = 64;                        // columns per chunk
  static constexpr int ST = 4;                         // pipeline stages
  static constexpr int ROWS = 8 * RW;                  // rows per CTA
  static constexpr size_t a_stage = size_t(8) * RW * CW * sizeof(CM);
  // LO: a second matrix tile (the low parts) per stage
  template <int NR, bool LO = false>
  static constexpr size_t smem() {
    return size_t(ST) * ((LO ? 2 : 1) * a_stage + size_t(NR) * CW * sizeof(CV));
  }
};
static_assert(GemvTile<float2, float2>::ROWS == 32 && GemvTile<double2, double2>::ROWS == 16, "tile rows");

template <int N>
__device__ __forceinline__ void cp_async_s(unsigned d, const void* src, bool valid) {  // shared address d
  const int n = valid ? N : 0;
  if constexpr (N == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
// packed FP32 pairs: (lo, hi) in one 64-bit register pair, d = a * b + d per component
__device__ __forceinline__ unsigned long long f32x2(float lo, float hi) {
  unsigned long long u;
  asm("mov.b64 %0, {%1, %2};" : "=l"(u) : "f"(lo), "f"(hi));
  return u;
}
__device__ __forceinline__ void f32x2_split(unsigned long long u, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(u));
}
__device__ __forceinline__ void ffma2(unsigned long long& d, unsigned long long a, unsigned long long b) {
  asm("fma.rn.f32x2 %0, %1, %2, %0;" : "+l"(d) : "l"(a), "l"(b));
}
// s + c += a1 b1 + a2 b2 + a1 b1lo + a2 b2lo, where b = b + blo is a split
// complex128 entry: the two main products are split exactly (product + FMA
// residual, Dekker / Kahan), the products enter s by TwoSum (Knuth; intrinsics
// keep the compiler from fusing or reordering), and every rounding error and
// low-order term gathers in c.  With s and c in FP32 the sum carries ~48 bits,
// on the FP32 pipe (64 x the FP64 rate of this part).
__device__ __forceinline__ void two_sum_into(float& s, float& c, float p) {
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, e);
}
__device__ __forceinline__ void comp_mac(float& s, float& c, float a1, float b1, float a2, float b2, float b1lo,
                                         float b2lo) {
  const float p1 = __fmul_rn(a1, b1), p2 = __fmul_rn(a2, b2);
  const float e1 = __fmaf_rn(a1, b1, -p1), e2 = __fmaf_rn(a2, b2, -p2);
  two_sum_into(s, c, p1);
  two_sum_into(s, c, p2);
  c = __fadd_rn(c, __fadd_rn(e1, e2));
  c = __fmaf_rn(a1, b1lo, c);
  c = __fmaf_rn(a2, b2lo, c);
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Sum v over the warp, C values per lane left, next exchange distance O.  When
// done lane l holds max(1, K/32) sums: value j is the total of index
// j + max(1, K/32) (l >> S), S = log2(32/K) for K < 32 and 0 otherwise.
template <int C, int O, class R, int K>
__device__ __forceinline__ void warp_tsum(R (&v)[K], int lane) {
  if constexpr (O > 0) {
    if constexpr (C >= 2) {
      const bool up = lane & O;
#pragma unroll
      for (int i = 0; i < C / 2; ++i) {
        const R send = up ? v[i] : v[i + C / 2];
        const R keep = up ? v[i + C / 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      warp_tsum<C / 2, O / 2>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], O);
      warp_tsum<C, O / 2>(v, lane);
    }
  }
}

// LO (complex64 blocks with complex128 vectors only): the job's Alo block streams
// beside A through the same pipeline, and its products with the high part of x
// join the error sum, so the result is that of the FP64 operator A + Alo.
template <class CM, class CV, int NR, bool LO = false>
__global__ void __launch_bounds__(256, LO ? 1 : 2) gemv_tile_kernel(const GemvJob* __restrict__ jobs,
                                                                   const int2* __restrict__ tiles, int nrhs, int col0) {
  typedef GemvTile<CM, CV> T;
  typedef typename CT<CV>::R R;
  constexpr int RW = T::RW, CW = T::CW, ST = T::ST;
  constexpr size_t a_all = (LO ? 2 : 1) * T::a_stage;     // matrix bytes per stage
  extern __shared__ __align__(16) unsigned char gsm[];
  CM* As = reinterpret_cast<CM*>(gsm);                     // [ST][8 warps][RW][2][32] (+ the same for Alo)
  CV* Xs = reinterpret_cast<CV*>(gsm + ST * a_all);        // [ST][NR][CW]
  const int2 t = tiles[blockIdx.x];
  const GemvJob J = jobs[t.x];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row0 = t.y + warp * RW;
  const CM* __restrict__ A = reinterpret_cast<const CM*>(J.A);
  const CM* __restrict__ Alo = reinterpret_cast<const CM*>(LO ? J.Alo : J.A);
  // right-hand sides col0 .. col0 + nrhs - 1 of the job's vectors
  const CV* __restrict__ x = reinterpret_cast<const CV*>(J.x) + int64_t(col0) * J.ldx;
  const int nch = (J.n + CW - 1) / CW;
  // per-thread copy sources (row 0 / right-hand side 0 stand in for rows or
  // right-hand sides outside the job: valid addresses, copied as zeros) and
  // shared-memory destinations in stage 0
  const CM* asrc[RW];
  int64_t aoff[RW];  // element offset of this lane's entry of row i (the same in Alo)
  bool arow[RW];
#pragma unroll
  for (int i = 0; i < RW; ++i) {
    arow[i] = row0 + i < J.m;
    aoff[i] = int64_t(arow[i] ? row0 + i : 0) * J.lda + lane;
    asrc[i] = A + aoff[i];
  }
  constexpr int XPT = (NR * CW + 255) / 256;  // x entries per thread per chunk
  const CV* xsrc[XPT];
  bool xok[XPT];
  int xcol[XPT];
#pragma unroll
  for (int q = 0; q < XPT; ++q) {
    const int e = q * 256 + threadIdx.x, r = e / CW;
    xcol[q] = e % CW;
    xok[q] = (NR * CW % 256 == 0 || e < NR * CW) && r < nrhs;
    xsrc[q] = x + (xok[q] ? int64_t(r) * J.ldx : 0) + xcol[q];
  }
  const unsigned a_dst = static_cast<unsigned>(__cvta_generic_to_shared(As + warp * RW * CW + lane));
  const unsigned x_dst = static_cast<unsigned>(__cvta_generic_to_shared(Xs + threadIdx.x));
  constexpr unsigned x_stage = NR * CW * sizeof(CV);
  auto issue = [&](int ch) {
    if (ch < nch) {
      const int st = ch & (ST - 1), c0 = ch * CW;
      const unsigned ad = a_dst + st * unsigned(a_all), xd = x_dst + st * x_stage;
      if (c0 + CW <= J.n) {  // a whole chunk: only row / right-hand-side validity
#pragma unroll
        for (int i = 0; i < RW; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            cp_async_s<sizeof(CM)>(ad + (i * 2 + j) * 32 * sizeof(CM), asrc[i] + c0 + j * 32, arow[i]);
            if constexpr (LO)
              cp_async_s<sizeof(CM)>(ad + unsigned(T::a_stage) + (i * 2 + j) * 32 * sizeof(CM), Alo + aoff[i] + c0 + j * 32,
                                     arow[i]);
          }
#pragma unroll
        for (int q = 0; q < XPT; ++q)
          if (NR * CW % 256 == 0 || q * 256 + int(threadIdx.x) < NR * CW)
            cp_async_s<sizeof(CV)>(xd + q * 256 * sizeof(CV), xsrc[q] + c0, xok[q]);
      } else {
#pragma unroll
        for (int i = 0; i < RW; ++i)
#pragma unroll
          for (int j = 0; j < 2; ++j) {
            const bool ok = arow[i] && c0 + j * 32 + lane < J.n;
            cp_async_s<sizeof(CM)>(ad + (i * 2 + j) * 32 * sizeof(CM), ok ? asrc[i] + c0 + j * 32 : A, ok);
            if constexpr (LO)
              cp_async_s<sizeof(CM)>(ad + unsigned(T::a_stage) + (i * 2 + j) * 32 * sizeof(CM),
                                     ok ? Alo + aoff[i] + c0 + j * 32 : Alo, ok);
          }
#pragma unroll
        for (int q = 0; q < XPT; ++q)
          if (NR * CW % 256 == 0 || q * 256 + int(threadIdx.x) < NR * CW) {
            const bool ok = xok[q] && c0 + xcol[q] < J.n;
            cp_async_s<sizeof(CV)>(xd + q * 256 * sizeof(CV), ok ? xsrc[q] + c0 : x, ok);
          }
      }
    }
    cp_commit();  // possibly empty: keeps one group per chunk
  };
#pragma unroll
  for (int c = 0; c < ST - 1; ++c) issue(c);
  constexpr bool PACKED = std::is_same<CM, float2>::value && std::is_same<CV, float2>::value;
  constexpr bool COMP = std::is_same<CM, float2>::value && std::is_same<CV, double2>::value;
  R acc[RW * NR * 2];
  unsigned long long acc2[PACKED ? RW * NR : 1];  // (re, im) pairs for the packed FP32 FMAs
  float cs[COMP ? RW * NR * 2 : 1], cc[COMP ? RW * NR * 2 : 1];  // compensated sums: value cs + cc
#pragma unroll
  for (int i = 0; i < RW * NR * 2; ++i) acc[i] = R(0);
#pragma unroll
  for (int i = 0; i < (PACKED ? RW * NR : 1); ++i) acc2[i] = 0ull;
#pragma unroll
  for (int i = 0; i < (COMP ? RW * NR * 2 : 1); ++i) cs[i] = cc[i] = 0.0f;
  for (int ch = 0; ch < nch; ++ch) {
    cp_wait<ST - 2>();  // this thread's copies of chunk ch have landed
    if constexpr (COMP) {
      // each thread splits the complex128 x entries it copied, in place, into
      // (hi, lo) complex64 pairs: x = hi + lo to 2^-48 relative
      CV* xs = Xs + (ch & (ST - 1)) * NR * CW;
#pragma unroll
      for (int q = 0; q < XPT; ++q)
        if (NR * CW % 256 == 0 || q * 256 + int(threadIdx.x) < NR * CW) {
          const double2 v = xs[q * 256 + threadIdx.x];
          const float hr = __double2float_rn(v.x), hi = __double2float_rn(v.y);
          reinterpret_cast<float4*>(xs)[q * 256 + threadIdx.x] =
              make_float4(hr, hi, __double2float_rn(v.x - double(hr)), __double2float_rn(v.y - double(hi)));
        }
    }
    __syncthreads();    // everyone's have, and chunk ch - 1 is consumed
    issue(ch + ST - 1); // into the slot of chunk ch - 1
    const int st = ch & (ST - 1);
    const CM* a = reinterpret_cast<const CM*>(gsm + st * a_all) + warp * RW * CW;
    const CM* alo = reinterpret_cast<const CM*>(gsm + st * a_all + T::a_stage) + warp * RW * CW;
    const CV* xs = Xs + st * NR * CW;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      CM av[RW];
#pragma unroll
      for (int i = 0; i < RW; ++i) av[i] = a[(i * 2 + j) * 32 + lane];
      if constexpr (PACKED) {
        // (acc_re, acc_im) += (a_re, a_re) (x_re, x_im) + (a_im, a_im) (-x_im, x_re):
        // the same two FMAs per component, in the same order, as cfma
        unsigned long long p1[RW], p2[RW];
#pragma unroll
        for (int i = 0; i < RW; ++i) {
          p1[i] = f32x2(float(av[i].x), float(av[i].x));
          p2[i] = f32x2(float(av[i].y), float(av[i].y));
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const CV xv = xs[r * CW + j * 32 + lane];
          const unsigned long long x1 = f32x2(float(xv.x), float(xv.y)), x2 = f32x2(-float(xv.y), float(xv.x));
#pragma unroll
          for (int i = 0; i < RW; ++i) {
            ffma2(acc2[i * NR + r], p1[i], x1);
            ffma2(acc2[i * NR + r], p2[i], x2);
          }
        }
      } else if constexpr (COMP) {
        CM lv[RW];
        if constexpr (LO) {
#pragma unroll
          for (int i = 0; i < RW; ++i) lv[i] = alo[(i * 2 + j) * 32 + lane];
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const float4 xv = reinterpret_cast<const float4*>(xs)[r * CW + j * 32 + lane];
#pragma unroll
          for (int i = 0; i < RW; ++i) {
            const int o = (i * NR + r) * 2;
            const float ar = float(av[i].x), ai = float(av[i].y);
            comp_mac(cs[o], cc[o], ar, xv.x, -ai, xv.y, xv.z, xv.w);      // re: ar xr - ai xi
            comp_mac(cs[o + 1], cc[o + 1], ar, xv.y, ai, xv.x, xv.w, xv.z);  // im: ar xi + ai xr
            if constexpr (LO) {  // + Alo x_hi: terms of 2^-24 relative, the rounding of their sum is below 2^-48
              const float lr = float(lv[i].x), li = float(lv[i].y);
              cc[o] = __fmaf_rn(lr, xv.x, __fmaf_rn(-li, xv.y, cc[o]));
              cc[o + 1] = __fmaf_rn(lr, xv.y, __fmaf_rn(li, xv.x, cc[o + 1]));
            }
          }
        }
      } else {
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          const CV xv = xs[r * CW + j * 32 + lane];
#pragma unroll
          for (int i = 0; i < RW; ++i)
            cfma(acc[(i * NR + r) * 2], acc[(i * NR + r) * 2 + 1], R(av[i].x), R(av[i].y), R(xv.x), R(xv.y));
        }
      }
    }
  }
  if constexpr (PACKED) {
#pragma unroll
    for (int i = 0; i < RW * NR; ++i) {
      float lo, hi;
      f32x2_split(acc2[i], lo, hi);
      acc[2 * i] = R(lo);
      acc[2 * i + 1] = R(hi);
    }
  }
  if constexpr (COMP) {
#pragma unroll
    for (int i = 0; i < RW * NR * 2; ++i) acc[i] = R(cs[i]) + R(cc[i]);
  }
  cp_wait<0>();
  constexpr int K = RW * NR * 2;
  constexpr int V = K >= 32 ? K / 32 : 1;
  constexpr int S = K >= 32 ? 0 : (K == 16 ? 1 : K == 8 ? 2 : K == 4 ? 3 : 4);
  warp_tsum<K, 16>(acc, lane);
  CV* y = reinterpret_cast<CV*>(J.y) + int64_t(col0) * J.ldy;
  auto put = [&](int p, R re, R im) {  // p = row-in-warp * NR + rhs
    const int i = p / NR, r = p % NR, row = row0 + i;
    if (row < J.m && r < nrhs) {
      R vr = R(J.ar) * re - R(J.ai) * im;
      R vi = R(J.ar) * im + R(J.ai) * re;
      CV* yy = y + int64_t(r) * J.ldy + row;
      if (J.beta) {
        vr += yy->x;
        vi += yy->y;
      }
      yy->x = vr;
      yy->y = vi;
    }
  };
  if constexpr (V >= 2) {
#pragma unroll
    for (int q = 0; q < V / 2; ++q) put((V / 2) * lane + q, acc[2 * q], acc[2 * q + 1]);
  } else {
    const R other = __shfl_xor_sync(0xffffffffu, acc[0], 1 << S);
    const int idx = lane >> S;
    if ((lane & ((1 << S) - 1)) == 0 && (idx & 1) == 0) put(idx >> 1, acc[0], other);
  }
}

template <class CM, class CV, int NR, bool LO = false>
static void launch_tile(const GemvPlan& plan, int nrhs, cudaStream_t s, int col0) {
  typedef GemvTile<CM, CV> T;
  constexpr size_t smem = T::template smem<NR, LO>();
  static_assert(smem <= 227 * 1024, "tile kernel exceeds the shared memory of one CTA");
  static std::atomic<uint64_t> done{0};  // devices whose attribute is set
  int dev = 0;
  SLDM_CUDA(cudaGetDevice(&dev));
  const uint64_t bit = uint64_t(1) << (dev & 63);
  if (!(done.load() & bit)) {
    SLDM_CUDA(cudaFuncSetAttribute(gemv_tile_kernel<CM, CV, NR, LO>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   int(smem)));
    done.fetch_or(bit);
  }
  gemv_tile_kernel<CM, CV, NR, LO><<<unsigned(plan.ntiles), 256, smem, s>>>(plan.jobs, plan.tiles, nrhs, col0);
  count_launch();
}

template <class CM, class CV>
void gemv_jobs_mixed(const GemvPlan& plan, int nrhs, cudaStream_t s) {
  if (plan.njobs == 0) return;
  const int64_t threads = plan.total_rows * 32;
  const unsigned blocks = unsigned((threads + 255) / 256);
  SLDM_REQUIRE(nrhs >= 1 && nrhs <= MAX_NRHS, SLDM_EINVAL, "GEMV: 1 to 32 right-hand sides per pass");
  constexpr bool comp = std::is_same<CM, float2>::value && std::is_same<CV, double2>::value;
  constexpr bool c64 = std::is_same<CM, float2>::value && std::is_same<CV, float2>::value;
  if constexpr (c64) {
    if (nrhs >= plan.tc_from && plan.tc != nullptr && plan.tc->ok) {  // one tensor-core pass
      ScopedTimer tm(plan.name, s);
      timer_units(plan.name, plan.bytes);
      gemm_tc(plan, *plan.tc, nrhs, s);
      return;
    }
  }
  ScopedTimer tm(plan.name, s);
  timer_units(plan.name, plan.bytes * double((nrhs + TILE_NRHS - 1) / TILE_NRHS));
  if (nrhs >= 2 || comp) {
    SLDM_REQUIRE((plan.tiles != nullptr && plan.tile_rows == GemvTile<CM, CV>::ROWS), SLDM_EINVAL,
                 "GEMV plan without row tiles for this vector type");
    if (plan.ntiles == 0) return;
    // passes of up to 8 right-hand sides on the CUDA cores
    for (int c0 = 0; c0 < nrhs; c0 += TILE_NRHS) {
      const int nr = std::min(TILE_NRHS, nrhs - c0);
      if constexpr (comp) {
        if (plan.has_lo) {  // the FP64 operator held as a complex64 pair
          if (nr <= 1) launch_tile<CM, CV, 1, true>(plan, nr, s, c0);
          else if (nr <= 2) launch_tile<CM, CV, 2, true>(plan, nr, s, c0);
          else if (nr <= 4) launch_tile<CM, CV, 4, true>(plan, nr, s, c0);
          else launch_tile<CM, CV, 8, true>(plan, nr, s, c0);
          continue;
        }
      }
      if (nr <= 1) {
        if constexpr (comp) launch_tile<CM, CV, 1>(plan, nr, s, c0);  // the only one-column use
        else launch_tile<CM, CV, 2>(plan, nr, s, c0);
      } else if (nr <= 2) launch_tile<CM, CV, 2>(plan, nr, s, c0);
      else if (nr <= 4) launch_tile<CM, CV, 4>(plan, nr, s, c0);
      else launch_tile<CM, CV, 8>(plan, nr, s, c0);
    }
  } else {
    gemv_jobs_kernel<CM, CV, 1><<<blocks, 256, 0, s>>>(plan.jobs, plan.rowstart, plan.njobs, plan.total_rows, nrhs);
    count_launch();
  }
  SLDM_CUDA(cudaGetLastError());
}
template void gemv_jobs_mixed<float2, double2>(const GemvPlan&, int, cudaStream_t);
template void gemv_jobs_mixed<float2, float2>(const GemvPlan&, int, cudaStream_t);
template void gemv_jobs_mixed<double2, double2>(const GemvPlan&, int, cudaStream_t);

static std::atomic<int> g_tc_force{0};  // sldm_set_tc_policy: 0 = measure, else the width to use

// decisions by plan shape (jobs, rows, bytes streamed per pass): a shape is timed once per process
static std::mutex g_tune_mu;
static std::map<std::tuple<int, int64_t, double>, int> g_tuned;

void gemv_autotune(GemvPlan& plan, cudaStream_t s) {
  if (plan.njobs == 0 || plan.tc == nullptr || !plan.tc->ok) return;
  if (const int f = g_tc_force.load()) {
    plan.tc_from = f;
    return;
  }
  const auto key = std::make_tuple(plan.njobs, plan.total_rows, plan.bytes);
  {
    std::lock_guard<std::mutex> l(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      plan.tc_from = it->second;
      return;
    }
  }
  cudaEvent_t e0, e1;
  SLDM_CUDA(cudaEventCreate(&e0));
  SLDM_CUDA(cudaEventCreate(&e1));
  auto timed = [&](int nrhs, int from) {
    plan.tc_from = from;
    gemv_jobs_mixed<float2, float2>(plan, nrhs, s);  // warm
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      SLDM_CUDA(cudaEventRecord(e0, s));
      gemv_jobs_mixed<float2, float2>(plan, nrhs, s);
      SLDM_CUDA(cudaEventRecord(e1, s));
      SLDM_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      SLDM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      best = std::min(best, ms);
    }
    return best;
  };
  timers_mute(true);  // keep the tuning passes out of the kernel timers
  float tc16 = 0, cc16 = 0, tc32 = 0, cc32 = 0;
  try {
    tc16 = timed(16, 1);
    cc16 = timed(16, MAX_NRHS + 1);
    tc32 = timed(32, 1);
    cc32 = timed(32, MAX_NRHS + 1);
  } catch (...) {
    timers_mute(false);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  timers_mute(false);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  plan.tc_from = tc16 < cc16 ? TILE_NRHS + 1 : (tc32 < cc32 ? 2 * TILE_NRHS + 1 : MAX_NRHS + 1);
  std::lock_guard<std::mutex> l(g_tune_mu);
  g_tuned[key] = plan.tc_from;
}


template <class C>
void gemv_jobs(const GemvPlan& plan, int nrhs, cudaStream_t s) {
  gemv_jobs_mixed<C, C>(plan, nrhs, s);
}

// ---------------------------------------------------------------- structured product glue
// x (complex128, N x nrhs) -> op precision split vectors j (ne), e (ne), u (nq) per rhs.
template <class C>
__global__ void split_in_kernel(const double2* __restrict__ x, int64_t ldx, int ne, int nq, C* j, C* e, C* u, int nrhs) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  int r = blockIdx.y;
  if (i >= 2 * ne + nq) return;
  double2 v = x[int64_t(r) * ldx + i];
  C c;
  c.x = decltype(c.x)(v.x);
  c.y = decltype(c.y)(v.y);
  if (i < ne) j[int64_t(r) * ne + i] = c;
  else if (i < 2 * ne) e[int64_t(r) * ne + (i - ne)] = c;
  else u[int64_t(r) * nq + (i - 2 * ne)] = c;
}

// a = j - t1 (ne);  c = u + t2 (nq);  bc = B c, bu = B u (nt), one CTA per (object, rhs)
template <class C>
__global__ void prep_kernel(const ApplyDims D, const int32_t* __restrict__ tri_begin, const int32_t* __restrict__ edge_begin,
                            const C* __restrict__ j, const C* __restrict__ u, const C* __restrict__ t1, const C* __restrict__ t2,
                            C* a, C* c, C* bc, C* bu) {
  typedef typename CT<C>::R R;
  const int o = blockIdx.x, r = blockIdx.y;
  const int t0 = tri_begin[o], t1e = tri_begin[o + 1];
  const int q0 = t0 - o, nq_o = t1e - t0 - 1;
  const int e0 = edge_begin[o], e1 = edge_begin[o + 1];
  const C* jr = j + int64_t(r) * D.ne;
  const C* t1r = t1 + int64_t(r) * D.ne;
  C* ar = a + int64_t(r) * D.ne;
  for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
    C v;
    v.x = jr[e].x - t1r[e].x;
    v.y = jr[e].y - t1r[e].y;
    ar[e] = v;
  }
  const C* ur = u + int64_t(r) * D.nq;
  const C* t2r = t2 + int64_t(r) * D.nq;
  C* cr = c + int64_t(r) * D.nq;
  C* bcr = bc + int64_t(r) * D.nt;
  C* bur = bu + int64_t(r) * D.nt;
  double sc_r = 0, sc_i = 0, su_r = 0, su_i = 0;
  for (int q = threadIdx.x; q < nq_o; q += blockDim.x) {
    C uv = ur[q0 + q];
    C v;
    v.x = uv.x + t2r[q0 + q].x;
    v.y = uv.y + t2r[q0 + q].y;
    cr[q0 + q] = v;
    bcr[t0 + q] = v;
    bur[t0 + q] = uv;
    sc_r += v.x;
    sc_i += v.y;
    su_r += uv.x;
    su_i += uv.y;
  }
  __shared__ double red[4][256];
  red[0][threadIdx.x] = sc_r;
  red[1][threadIdx.x] = sc_i;
  red[2][threadIdx.x] = su_r;
  red[3][threadIdx.x] = su_i;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w)
      for (int k = 0; k < 4; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    C v;
    v.x = R(-red[0][0]);
    v.y = R(-red[1][0]);
    bcr[t1e - 1] = v;
    v.x = R(-red[2][0]);
    v.y = R(-red[3][0]);
    bur[t1e - 1] = v;
  }
}

// y1 = z1 + D^T z2 + I_x e;  y2 = w1 - w2 + D^T w3;  y3 = F D a + k0^2 c   (complex128 output)
template <class C>
__global__ void combine_kernel(const ApplyDims D, double k0, const int32_t* __restrict__ tplus, const int32_t* __restrict__ tminus,
                               const int32_t* __restrict__ tri_edge, const int8_t* __restrict__ tri_sign,
                               const int32_t* __restrict__ q2t, const int32_t* __restrict__ ix_ptr,
                               const int32_t* __restrict__ ix_col, const double* __restrict__ ix_val, const C* __restrict__ z1,
                               const C* __restrict__ z2, const C* __restrict__ w1, const C* __restrict__ w2,
                               const C* __restrict__ w3, const C* __restrict__ e, const C* __restrict__ a,
                               const C* __restrict__ c, double2* y, int64_t ldy) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  const int ne = D.ne, nt = D.nt, nq = D.nq;
  if (i >= 2 * ne + nq) return;
  double vr, vi;
  if (i < ne) {
    const int m = int(i);
    C a1 = z1[int64_t(r) * ne + m];
    C p = z2[int64_t(r) * nt + tplus[m]], q = z2[int64_t(r) * nt + tminus[m]];
    vr = double(a1.x) + double(p.x) - double(q.x);
    vi = double(a1.y) + double(p.y) - double(q.y);
    for (int z = ix_ptr[m]; z < ix_ptr[m + 1]; ++z) {
      C ev = e[int64_t(r) * ne + ix_col[z]];
      vr += ix_val[z] * double(ev.x);
      vi += ix_val[z] * double(ev.y);
    }
  } else if (i < 2 * ne) {
    const int m = int(i - ne);
    C a1 = w1[int64_t(r) * ne + m], b1 = w2[int64_t(r) * ne + m];
    C p = w3[int64_t(r) * nt + tplus[m]], q = w3[int64_t(r) * nt + tminus[m]];
    vr = double(a1.x) - double(b1.x) + double(p.x) - double(q.x);
    vi = double(a1.y) - double(b1.y) + double(p.y) - double(q.y);
  } else {
    const int qq = int(i - 2 * ne);
    const int t = q2t[qq];  // triangle of charge unknown qq (each object's last triangle has none)
    double sr = 0, si = 0;
    for (int k = 0; k < 3; ++k) {
      C av = a[int64_t(r) * ne + tri_edge[3 * t + k]];
      double sg = double(tri_sign[3 * t + k]);
      sr += sg * double(av.x);
      si += sg * double(av.y);
    }
    C cv = c[int64_t(r) * nq + qq];
    vr = sr + k0 * k0 * double(cv.x);
    vi = si + k0 * k0 * double(cv.y);
  }
  y[int64_t(r) * ldy + i] = make_double2(vr, vi);
}

template <class C>
void apply_glue_split(const double2* x, int64_t ldx, const ApplyDims& D, void* j, void* e, void* u, int nrhs, cudaStream_t s) {
  int64_t N = 2 * D.ne + D.nq;
  split_in_kernel<C><<<dim3(unsigned((N + 255) / 256), nrhs), 256, 0, s>>>(x, ldx, D.ne, D.nq, (C*)j, (C*)e, (C*)u, nrhs), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

template <class C>
void apply_glue_prep(const sldm_mesh* m, const ApplyDims& D, const void* j, const void* u, const void* t1, const void* t2,
                     void* a, void* c, void* bc, void* bu, int nrhs, cudaStream_t s, const int32_t* tri_begin_dev,
                     const int32_t* edge_begin_dev) {
  prep_kernel<C><<<dim3(unsigned(D.nobj), nrhs), 256, 0, s>>>(D, tri_begin_dev, edge_begin_dev, (const C*)j, (const C*)u,
                                                             (const C*)t1, (const C*)t2, (C*)a, (C*)c, (C*)bc, (C*)bu), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

template <class C>
void apply_glue_combine(const sldm_mesh* m, const ApplyDims& D, double k0, const double* ix_val, const void* z1,
                        const void* z2, const void* w1, const void* w2, const void* w3, const void* e, const void* a,
                        const void* c, double2* y, int64_t ldy, int nrhs, cudaStream_t s) {
  int64_t N = 2 * D.ne + D.nq;
  const DevMesh& d = m->d;
  combine_kernel<C><<<dim3(unsigned((N + 255) / 256), nrhs), 256, 0, s>>>(
      D, k0, d.tplus.p, d.tminus.p, d.tri_edge.p, d.tri_sign.p, d.q2t.p, d.ix_ptr.p, d.ix_col.p, ix_val, (const C*)z1,
      (const C*)z2, (const C*)w1, (const C*)w2, (const C*)w3, (const C*)e, (const C*)a, (const C*)c, y, ldy), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// ---------------------------------------------------------------- vector kernels for GMRES
// Templated on the storage of the Krylov basis and of the vector being
// orthogonalised: complex128 (FP64 arithmetic) for complex128 operators,
// complex64 (FP32 arithmetic, FP64 sums across threads) for complex64 ones.
// On this part FP64 issues at 1/64 of the FP32 rate, so an FP64 dot product
// or update (4 FMAs per complex entry) tops out near 2.5 TB/s of complex128
// entries, below HBM; in complex64 the same kernels are HBM-bound.
template <class C>
__device__ __forceinline__ C cmake(double x, double y);
template <>
__device__ __forceinline__ float2 cmake<float2>(double x, double y) { return make_float2(float(x), float(y)); }
template <>
__device__ __forceinline__ double2 cmake<double2>(double x, double y) { return make_double2(x, y); }

// w += sign * V[:, :k] h (arithmetic in w's precision).  A CTA owns 32 rows;
// its 8 warps take every 8th Krylov column, four columns in flight, and the
// partial sums meet in shared memory.
template <class CB, class CW>
__global__ void __launch_bounds__(256) vmul_kernel(const CB* __restrict__ V, int64_t ldv, int k,
                                                   const double2* __restrict__ h, double sign, CW* w, int64_t n) {
  typedef typename CT<CW>::R R;
  __shared__ R part[8][32][2];
  const int lane = threadIdx.x & 31, slice = threadIdx.x >> 5;
  const int64_t t = int64_t(blockIdx.x) * 32 + lane;
  R sr = 0, si = 0;
  if (t < n) {
    int i = slice;
    for (; i + 24 < k; i += 32) {
      CB v[4];
      double2 c[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        v[u] = V[int64_t(i + 8 * u) * ldv + t];
        c[u] = h[i + 8 * u];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) cfma(sr, si, R(v[u].x), R(v[u].y), R(c[u].x), R(c[u].y));
    }
    for (; i < k; i += 8) {
      const CB v = V[int64_t(i) * ldv + t];
      const double2 c = h[i];
      cfma(sr, si, R(v.x), R(v.y), R(c.x), R(c.y));
    }
  }
  part[slice][lane][0] = sr;
  part[slice][lane][1] = si;
  __syncthreads();
  if (slice == 0 && t < n) {
    R ar = 0, ai = 0;
    for (int q = 0; q < 8; ++q) {
      ar += part[q][lane][0];
      ai += part[q][lane][1];
    }
    const CW o = w[t];
    w[t].x = o.x + R(sign) * ar;
    w[t].y = o.y + R(sign) * ai;
  }
}

template <class C>
__global__ void norm2_kernel(const C* __restrict__ w, int64_t n, double* out) {
  double s = 0;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += int64_t(gridDim.x) * blockDim.x) {
    const C a = w[t];
    s += double(a.x) * double(a.x) + double(a.y) * double(a.y);
  }
  __shared__ double r[256];
  r[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) r[threadIdx.x] += r[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(out, r[0]);
}

// y = alpha * x + beta * y (real alpha, beta; FP64 arithmetic, y stored in its type;
// beta = 0 ignores the old y)
template <class CX, class CY>
__global__ void axpby_kernel(int64_t n, double alpha, const CX* __restrict__ x, double beta, CY* y) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const CX a = x[t];
  double vr = alpha * double(a.x), vi = alpha * double(a.y);
  if (beta != 0.0) {
    const CY b = y[t];
    vr += beta * double(b.x);
    vi += beta * double(b.y);
  }
  y[t] = cmake<CY>(vr, vi);
}

// y[i] = s_b x[i] with s_b = s1 on [0, ne), s2 on [ne, 2 ne), s3 on [2 ne, n) (in place allowed)
template <class CX, class CY>
__global__ void vscale3_kernel(int64_t n, int64_t ne, double s1, double s2, double s3, const CX* __restrict__ x, CY* y) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const double s = t < ne ? s1 : (t < 2 * ne ? s2 : s3);
  const CX a = x[t];
  y[t] = cmake<CY>(s * double(a.x), s * double(a.y));
}

template <class CX, class CY>
void vscale3(int64_t n, int64_t ne, double s1, double s2, double s3, const CX* x, CY* y, cudaStream_t s) {
  vscale3_kernel<CX, CY><<<unsigned((n + 255) / 256), 256, 0, s>>>(n, ne, s1, s2, s3, x, y), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template <class CB, class CW>
void vmul(const CB* V, int64_t ldv, int k, const double2* h, double sign, CW* w, int64_t n, cudaStream_t s) {
  vmul_kernel<CB, CW><<<unsigned((n + 31) / 32), 256, 0, s>>>(V, ldv, k, h, sign, w, n), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template <class C>
void vnorm2(const C* w, int64_t n, double* out, cudaStream_t s) {
  SLDM_CUDA(cudaMemsetAsync(out, 0, sizeof(double), s));
  unsigned b = unsigned(std::min<int64_t>((n + 255) / 256, 1024));
  norm2_kernel<C><<<b, 256, 0, s>>>(w, n, out), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template <class CX, class CY>
void vaxpby(int64_t n, double alpha, const CX* x, double beta, CY* y, cudaStream_t s) {
  axpby_kernel<CX, CY><<<unsigned((n + 255) / 256), 256, 0, s>>>(n, alpha, x, beta, y), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
#define SLDM_VEC_INST(CX, CY)                                                                                   \
  template void vscale3<CX, CY>(int64_t, int64_t, double, double, double, const CX*, CY*, cudaStream_t);       \
  template void vmul<CX, CY>(const CX*, int64_t, int, const double2*, double, CY*, int64_t, cudaStream_t);     \
  template void vaxpby<CX, CY>(int64_t, double, const CX*, double, CY*, cudaStream_t);
SLDM_VEC_INST(double2, double2)
SLDM_VEC_INST(float2, float2)
SLDM_VEC_INST(float2, double2)
SLDM_VEC_INST(double2, float2)
#undef SLDM_VEC_INST
template void vnorm2<double2>(const double2*, int64_t, double*, cudaStream_t);
template void vnorm2<float2>(const float2*, int64_t, double*, cudaStream_t);

// ---------------------------------------------------------------- batched Gram-Schmidt
// One launch per pass for every live right-hand side of a lockstep step.  The
// bases have a column stride ldv that is a multiple of 64 entries and zero
// rows from n up to ldv, so every lane handles two consecutive rows (one
// 16-byte load in complex64) with no tail.
__device__ __forceinline__ void ld_pair(const float2* p, float2& a, float2& b) {
  const float4 q = *reinterpret_cast<const float4*>(p);
  a = make_float2(q.x, q.y);
  b = make_float2(q.z, q.w);
}
__device__ __forceinline__ void ld_pair(const double2* p, double2& a, double2& b) {
  a = p[0];
  b = p[1];
}
__device__ __forceinline__ void st_pair(float2* p, float2 a, float2 b) {
  *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_pair(double2* p, double2 a, double2 b) {
  p[0] = a;
  p[1] = b;
}

// h_j[i] += V_j[:, i]^H V_j[:, k] for i < k.  Grid (ceil(k / 8), row chunks, na):
// warp i % 8 of a CTA takes column i over the CTA's KRYLOV_CHUNK rows.
constexpr int KRYLOV_CHUNK = 2048;
template <class CB>
__global__ void __launch_bounds__(256) krylov_dots_kernel(KrylovStep ks) {
  typedef typename CT<CB>::R R;
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (i >= ks.k) return;
  const CB* V = reinterpret_cast<const CB*>(ks.V[blockIdx.z]);
  const CB* __restrict__ v = V + int64_t(i) * ks.ldv;
  const CB* __restrict__ w = V + int64_t(ks.k) * ks.ldv;
  const int64_t r0 = int64_t(blockIdx.y) * KRYLOV_CHUNK;
  const int64_t r1 = r0 + KRYLOV_CHUNK < ks.ldv ? r0 + KRYLOV_CHUNK : ks.ldv;
  R sr = 0, si = 0, tr = 0, ti = 0;
#pragma unroll 4
  for (int64_t t = r0 + 2 * lane; t < r1; t += 64) {
    CB a0, a1, b0, b1;
    ld_pair(v + t, a0, a1);
    ld_pair(w + t, b0, b1);
    cfma(sr, si, a0.x, -a0.y, b0.x, b0.y);  // conj(a) b
    cfma(tr, ti, a1.x, -a1.y, b1.x, b1.y);
  }
  double dr = double(sr) + double(tr), di = double(si) + double(ti);
  for (int o = 16; o > 0; o >>= 1) {
    dr += __shfl_xor_sync(0xffffffffu, dr, o);
    di += __shfl_xor_sync(0xffffffffu, di, o);
  }
  if (lane == 0) {
    atomicAdd(&ks.h[blockIdx.z][i].x, dr);
    atomicAdd(&ks.h[blockIdx.z][i].y, di);
  }
}

// V_j[:, k] -= V_j[:, :k] h_j, and with `norm` nrm[j] += |V_j[:, k]|^2 after the
// update.  Grid (ldv / 512, na): warp = 64 rows (lane = 2), over all k columns
// with eight column loads in flight and no exchange between warps.
template <class CB>
__global__ void __launch_bounds__(256) krylov_update_kernel(KrylovStep ks, int norm) {
  typedef typename CT<CB>::R R;
  const int lane = threadIdx.x & 31;
  const int64_t r0 = (int64_t(blockIdx.x) * 8 + (threadIdx.x >> 5)) * 64;
  if (r0 >= ks.ldv) return;  // whole warps
  const int j = blockIdx.y;
  CB* V = reinterpret_cast<CB*>(ks.V[j]);
  const double2* __restrict__ h = ks.h[j];
  const int64_t t = r0 + 2 * lane;
  R s0r = 0, s0i = 0, s1r = 0, s1i = 0;
  int i = 0;
  for (; i + 8 <= ks.k; i += 8) {
    CB a[8], b[8];
    double2 c[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      ld_pair(V + int64_t(i + u) * ks.ldv + t, a[u], b[u]);
      c[u] = h[i + u];
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      cfma(s0r, s0i, R(a[u].x), R(a[u].y), R(c[u].x), R(c[u].y));
      cfma(s1r, s1i, R(b[u].x), R(b[u].y), R(c[u].x), R(c[u].y));
    }
  }
  for (; i < ks.k; ++i) {
    CB a, b;
    ld_pair(V + int64_t(i) * ks.ldv + t, a, b);
    const double2 c = h[i];
    cfma(s0r, s0i, R(a.x), R(a.y), R(c.x), R(c.y));
    cfma(s1r, s1i, R(b.x), R(b.y), R(c.x), R(c.y));
  }
  CB* w = V + int64_t(ks.k) * ks.ldv + t;
  CB a, b;
  ld_pair(w, a, b);
  a.x -= s0r;
  a.y -= s0i;
  b.x -= s1r;
  b.y -= s1i;
  st_pair(w, a, b);
  if (norm) {
    double nn = double(a.x) * double(a.x) + double(a.y) * double(a.y) + double(b.x) * double(b.x) + double(b.y) * double(b.y);
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) atomicAdd(ks.nrm + j, nn);
  }
}

template <class CB>
void krylov_dots(const KrylovStep& ks, cudaStream_t s) {
  if (ks.k <= 0 || ks.na <= 0) return;
  krylov_dots_kernel<CB><<<dim3(unsigned((ks.k + 7) / 8), unsigned((ks.ldv + KRYLOV_CHUNK - 1) / KRYLOV_CHUNK), ks.na), 256, 0,
                           s>>>(ks), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template <class CB>
void krylov_update(const KrylovStep& ks, bool norm, cudaStream_t s) {
  if (ks.na <= 0) return;
  krylov_update_kernel<CB><<<dim3(unsigned((ks.ldv / 64 + 7) / 8), ks.na), 256, 0, s>>>(ks, norm ? 1 : 0),
      ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template void krylov_dots<float2>(const KrylovStep&, cudaStream_t);
template void krylov_dots<double2>(const KrylovStep&, cudaStream_t);
template void krylov_update<float2>(const KrylovStep&, bool, cudaStream_t);
template void krylov_update<double2>(const KrylovStep&, bool, cudaStream_t);

// y_j = a_j s(i) x_j[i] for the na column pairs, s = s1, s2, s3 on the three blocks
template <class CX, class CY>
__global__ void vscale3_batch_kernel(int64_t n, int64_t ne, double s1, double s2, double s3, VecBatch<CX, CY> b) {
  const int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int j = blockIdx.y;
  const double sc = b.a[j] * (t < ne ? s1 : (t < 2 * ne ? s2 : s3));
  const CX v = b.x[j][t];
  b.y[j][t] = cmake<CY>(sc * double(v.x), sc * double(v.y));
}
template <class CX, class CY>
void vscale3_batch(int64_t n, int64_t ne, double s1, double s2, double s3, const VecBatch<CX, CY>& b, int na,
                   cudaStream_t s) {
  if (na <= 0) return;
  vscale3_batch_kernel<CX, CY><<<dim3(unsigned((n + 255) / 256), na), 256, 0, s>>>(n, ne, s1, s2, s3, b), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template void vscale3_batch<double2, double2>(int64_t, int64_t, double, double, double, const VecBatch<double2, double2>&, int,
                                              cudaStream_t);
template void vscale3_batch<float2, double2>(int64_t, int64_t, double, double, double, const VecBatch<float2, double2>&, int,
                                             cudaStream_t);
template void vscale3_batch<double2, float2>(int64_t, int64_t, double, double, double, const VecBatch<double2, float2>&, int,
                                             cudaStream_t);
template void vscale3_batch<float2, float2>(int64_t, int64_t, double, double, double, const VecBatch<float2, float2>&, int,
                                            cudaStream_t);

// ---------------------------------------------------------------- conversions
template <class C>
__global__ void to_c128_kernel(const C* __restrict__ src, int64_t n, double2* dst) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) dst[t] = make_double2(double(src[t].x), double(src[t].y));
}
template <class C>
__global__ void from_c128_kernel(const double2* __restrict__ src, int64_t n, C* dst) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t < n) {
    dst[t].x = decltype(dst[t].x)(src[t].x);
    dst[t].y = decltype(dst[t].y)(src[t].y);
  }
}
template <class C>
void to_c128(const void* src, int64_t n, double2* dst, cudaStream_t s) {
  to_c128_kernel<C><<<unsigned((n + 255) / 256), 256, 0, s>>>((const C*)src, n, dst), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template <class C>
void from_c128(const double2* src, int64_t n, void* dst, cudaStream_t s) {
  from_c128_kernel<C><<<unsigned((n + 255) / 256), 256, 0, s>>>(src, n, (C*)dst), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// FP64 operator kept as a complex64 pair: hi = fl32(v), lo = fl32(v - hi)
__global__ void split_c128_kernel(const double2* __restrict__ src, int64_t n, float2* __restrict__ hi,
                                  float2* __restrict__ lo) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
    const double2 v = src[t];
    const float hr = __double2float_rn(v.x), hv = __double2float_rn(v.y);
    hi[t] = make_float2(hr, hv);
    lo[t] = make_float2(__double2float_rn(v.x - double(hr)), __double2float_rn(v.y - double(hv)));
  }
}
__global__ void add_lo_c128_kernel(const float2* __restrict__ lo, int64_t n, double2* dst) {
  const int64_t stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; t < n; t += stride) {
    dst[t].x += double(lo[t].x);
    dst[t].y += double(lo[t].y);
  }
}
void split_c128(const double2* src, int64_t n, float2* hi, float2* lo, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned blocks = unsigned(std::min<int64_t>((n + 255) / 256, 152 * 32));
  split_c128_kernel<<<blocks, 256, 0, s>>>(src, n, hi, lo), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
void add_lo_c128(const float2* lo, int64_t n, double2* dst, cudaStream_t s) {
  if (n <= 0) return;
  const unsigned blocks = unsigned(std::min<int64_t>((n + 255) / 256, 152 * 32));
  add_lo_c128_kernel<<<blocks, 256, 0, s>>>(lo, n, dst), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// One warp per copied row: the rows of every copy, in order, split by an
// exclusive prefix sum; 16-byte loads when the entries are complex128 or the
// row segment is 16-byte aligned.
template <class C>
__global__ void __launch_bounds__(256) copy_blocks_kernel(const BlockCopy* __restrict__ cp, const int64_t* __restrict__ rs,
                                                          int ncp, int64_t total_rows, C* M, int64_t ld) {
  const int64_t w = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= total_rows) return;
  int lo = 0, hi = ncp - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (rs[mid] <= w) lo = mid;
    else hi = mid - 1;
  }
  const BlockCopy c = cp[lo];
  const int64_t r = w - rs[lo];
  const C* src = M + (c.sr + r) * ld + c.sc;
  C* dst = M + (c.dr + r) * ld + c.dc;
  for (int j = lane; j < c.nc; j += 32) dst[j] = __ldcs(src + j);
}

void copy_blocks(const std::vector<BlockCopy>& copies, size_t esz, void* M, int64_t ld, cudaStream_t s) {
  if (copies.empty()) return;
  std::vector<int64_t> rs(copies.size());
  int64_t acc = 0;
  for (size_t i = 0; i < copies.size(); ++i) {
    rs[i] = acc;
    acc += copies[i].nr;
  }
  DBuf<BlockCopy> dc;
  DBuf<int64_t> drs;
  dc.upload(copies, s);
  drs.upload(rs, s);
  const unsigned blocks = unsigned((acc * 32 + 255) / 256);
  ScopedTimer tm("copy_blocks", s);
  if (esz == sizeof(double2))
    copy_blocks_kernel<double2><<<blocks, 256, 0, s>>>(dc.p, drs.p, int(copies.size()), acc, (double2*)M, ld);
  else
    copy_blocks_kernel<float2><<<blocks, 256, 0, s>>>(dc.p, drs.p, int(copies.size()), acc, (float2*)M, ld);
  count_launch();
  SLDM_CUDA(cudaGetLastError());
  SLDM_CUDA(cudaStreamSynchronize(s));  // the copy lists are released on return
}

// add alpha * I_x (CSR, rows of an object) into a dense block
template <class C>
__global__ void add_ix_kernel(int e0, int ne_o, double alpha, const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                              const double* __restrict__ val, C* K, int64_t ld) {
  int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= ne_o) return;
  for (int z = ptr[e0 + m]; z < ptr[e0 + m + 1]; ++z) {
    int n = col[z] - e0;
    if (n >= 0 && n < ne_o) {
      K[int64_t(m) * ld + n].x += decltype(K[0].x)(alpha * val[z]);
    }
  }
}
template <class C>
void add_ix(const sldm_mesh* m, int obj, double alpha, const double* ix_val, void* K, int64_t ld, cudaStream_t s) {
  int e0 = m->h.edge_begin[obj], ne_o = m->h.edge_begin[obj + 1] - e0;
  add_ix_kernel<C><<<(ne_o + 127) / 128, 128, 0, s>>>(e0, ne_o, alpha, m->d.ix_ptr.p, m->d.ix_col.p, ix_val, (C*)K, ld), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// dst = alpha * src (real alpha)
template <class C>
__global__ void copy_scaled_kernel(const C* __restrict__ src, int64_t n, double alpha, C* dst) {
  int64_t t = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (t >= n) return;
  C v = src[t];
  v.x = decltype(v.x)(double(v.x) * alpha);
  v.y = decltype(v.y)(double(v.y) * alpha);
  dst[t] = v;
}
template <class C>
void copy_scaled(const void* src, int64_t n, double alpha, void* dst, cudaStream_t s) {
  if (n <= 0) return;
  copy_scaled_kernel<C><<<unsigned((n + 255) / 256), 256, 0, s>>>((const C*)src, n, alpha, (C*)dst), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

#define INST(C)                                                                                                         \
  template void build_Ml<C>(const sldm_mesh*, int, double, const void*, int64_t, const void*, int64_t, const void*,     \
                            int64_t, const double*, C*, C*, cudaStream_t);                                              \
  template void gemv_jobs<C>(const GemvPlan&, int, cudaStream_t);                                                       \
  template void apply_glue_split<C>(const double2*, int64_t, const ApplyDims&, void*, void*, void*, int, cudaStream_t); \
  template void apply_glue_prep<C>(const sldm_mesh*, const ApplyDims&, const void*, const void*, const void*,           \
                                   const void*, void*, void*, void*, void*, int, cudaStream_t, const int32_t*,         \
                                   const int32_t*);                                                                     \
  template void apply_glue_combine<C>(const sldm_mesh*, const ApplyDims&, double, const double*, const void*,           \
                                      const void*, const void*, const void*, const void*, const void*, const void*,     \
                                      const void*, double2*, int64_t, int, cudaStream_t);                               \
  template void to_c128<C>(const void*, int64_t, double2*, cudaStream_t);                                               \
  template void from_c128<C>(const double2*, int64_t, void*, cudaStream_t);                                             \
  template void add_ix<C>(const sldm_mesh*, int, double, const double*, void*, int64_t, cudaStream_t);             \
  template void copy_scaled<C>(const void*, int64_t, double, void*, cudaStream_t);
INST(float2)
INST(double2)

// ---------------------------------------------------------------- GMRES on the device
__device__ __forceinline__ double2 zmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ __forceinline__ double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double zabs(double2 a) { return hypot(a.x, a.y); }

// One warp per active right-hand side: the lanes stage column k of H and the
// earlier rotations in shared memory, lane 0 applies the rotations in order (each
// depends on the previous one) and the new one, and the lanes write the column back.
__global__ void gmres_givens_kernel(GivensArgs a) {
  extern __shared__ __align__(16) unsigned char gv_raw[];
  double2* gsm = reinterpret_cast<double2*>(gv_raw);  // column (m + 2), cs (m), sn (m)
  const int j = blockIdx.x;
  if (j >= a.na) return;
  const int r = a.on[j];
  GmresState* st = a.st + r;
  const int lane = threadIdx.x;
  if (!st->live) {
    if (lane == 0) a.scale[j] = 0.0;
    return;
  }
  const int m = a.m, k = a.k;
  const double2* hr = a.dh + int64_t(r) * a.ldh;
  double2* H = a.H + int64_t(r) * (m + 1) * m;
  double2* cs = a.cs + int64_t(r) * m;
  double2* sn = a.sn + int64_t(r) * m;
  double2* g = a.g + int64_t(r) * (m + 1);
  double2* col = gsm;
  double2* scs = gsm + (m + 2);
  double2* ssn = scs + m;
  const double h1 = sqrt(a.nrm[j]);
  for (int i = lane; i <= k; i += 32) col[i] = zadd(hr[i], hr[(m + 2) + i]);
  for (int i = lane; i < k; i += 32) {
    scs[i] = cs[i];
    ssn[i] = sn[i];
  }
  if (lane == 0) col[k + 1] = make_double2(h1, 0.0);
  __syncwarp();
  if (lane == 0) {
    for (int i = 0; i < k; ++i) {  // the earlier rotations
      const double2 x = col[i], y = col[i + 1];
      col[i] = zadd(zmul(scs[i], x), zmul(ssn[i], y));
      const double2 msn = zconj(ssn[i]);
      col[i + 1] = zadd(make_double2(-(msn.x * x.x - msn.y * x.y), -(msn.x * x.y + msn.y * x.x)), zmul(scs[i], y));
    }
    const double2 x = col[k], y = col[k + 1];
    const double ax = zabs(x);
    const double t = sqrt(x.x * x.x + x.y * x.y + y.x * y.x + y.y * y.y);
    double2 c, sv;
    if (ax == 0) {
      c = make_double2(0.0, 0.0);
      sv = make_double2(1.0, 0.0);
      col[k] = y;
    } else {
      const double2 ph = make_double2(x.x / ax, x.y / ax);  // a / |a|
      c = make_double2(ax / t, 0.0);
      const double2 p = zmul(ph, zconj(y));
      sv = make_double2(p.x / t, p.y / t);
      col[k] = make_double2(ph.x * t, ph.y * t);
    }
    col[k + 1] = make_double2(0.0, 0.0);
    cs[k] = c;
    sn[k] = sv;
    const double2 gk = g[k];
    const double2 msn = zconj(sv);
    g[k + 1] = make_double2(-(msn.x * gk.x - msn.y * gk.y), -(msn.x * gk.y + msn.y * gk.x));
    g[k] = zmul(c, gk);
    st->it += 1;
    st->kused = k + 1;
    const double res = zabs(g[k + 1]);
    if (res / st->bnorm <= a.tol || st->it >= a.maxit || h1 == 0) st->live = 0;
    if (a.refine && res <= a.cycle * st->beta) st->live = 0;
    a.scale[j] = h1 > 0 ? 1.0 / h1 : 0.0;
  }
  __syncwarp();
  for (int i = lane; i <= k + 1; i += 32) H[int64_t(i) * m + k] = col[i];
}

void gmres_givens(const GivensArgs& a, cudaStream_t s) {
  if (a.na <= 0) return;
  const size_t smem = size_t(3 * a.m + 2) * sizeof(double2);
  SLDM_REQUIRE(smem <= 48 * 1024, SLDM_EINVAL, "GMRES: restart length too large for the device rotations");
  gmres_givens_kernel<<<a.na, 32, smem, s>>>(a), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

// one warp per right-hand side: back substitution, row by row from the bottom,
// the sum over the columns to the right split across the lanes
__global__ void gmres_backsolve_kernel(int na, const int* __restrict__ on, int m, const double2* __restrict__ H,
                                       const double2* __restrict__ g, const GmresState* __restrict__ st, double2* dh,
                                       int64_t ldh) {
  const int j = blockIdx.x;
  if (j >= na) return;
  const int r = on[j];
  const int ku = st[r].kused;
  const double2* Hr = H + int64_t(r) * (m + 1) * m;
  const double2* gr = g + int64_t(r) * (m + 1);
  double2* y = dh + int64_t(r) * ldh;
  const int lane = threadIdx.x;
  for (int i = ku - 1; i >= 0; --i) {
    double sr = 0, si = 0;
    for (int c = i + 1 + lane; c < ku; c += 32) {
      const double2 h = Hr[int64_t(i) * m + c], v = y[c];
      sr += h.x * v.x - h.y * v.y;
      si += h.x * v.y + h.y * v.x;
    }
    for (int o = 16; o > 0; o >>= 1) {
      sr += __shfl_down_sync(0xffffffffu, sr, o);
      si += __shfl_down_sync(0xffffffffu, si, o);
    }
    if (lane == 0) {
      const double2 acc = make_double2(gr[i].x - sr, gr[i].y - si);
      const double2 d = Hr[int64_t(i) * m + i];
      const double dn = d.x * d.x + d.y * d.y;
      y[i] = make_double2((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn);
    }
    __syncwarp();
  }
}

void gmres_backsolve(int na, const int* on, int m, const double2* H, const double2* g, const GmresState* st, double2* dh,
                     int64_t ldh, cudaStream_t s) {
  if (na <= 0) return;
  gmres_backsolve_kernel<<<na, 32, 0, s>>>(na, on, m, H, g, st, dh, ldh), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}

template <class CB>
__global__ void vscale_dev_kernel(int64_t n, VecBatch<CB, CB> b, const double* __restrict__ scale) {
  const int j = blockIdx.y;
  const double a = scale[j];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    CB v = b.x[j][i];
    v.x = decltype(v.x)(double(v.x) * a);
    v.y = decltype(v.y)(double(v.y) * a);
    b.y[j][i] = v;
  }
}

template <class CB>
void vscale_dev_batch(int64_t n, const VecBatch<CB, CB>& b, const double* scale, int na, cudaStream_t s) {
  if (na <= 0) return;
  const unsigned gx = unsigned(std::min<int64_t>((n + 255) / 256, 1024));
  vscale_dev_kernel<CB><<<dim3(gx, na), 256, 0, s>>>(n, b, scale), ::sldm::count_launch();
  SLDM_CUDA(cudaGetLastError());
}
template void vscale_dev_batch<double2>(int64_t, const VecBatch<double2, double2>&, const double*, int, cudaStream_t);
template void vscale_dev_batch<float2>(int64_t, const VecBatch<float2, float2>&, const double*, int, cudaStream_t);

}  // namespace sldm

extern "C" int sldm_set_tc_policy(int32_t tc_from) {
  if (tc_from != 0 && (tc_from < 1 || tc_from > sldm::MAX_NRHS + 1)) return SLDM_EINVAL;
  sldm::g_tc_force.store(tc_from);
  return SLDM_OK;
}
