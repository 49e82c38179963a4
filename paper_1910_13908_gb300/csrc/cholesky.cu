// Step (c, solve): dense Cholesky factorisation A = L L^T of the damped
// Gauss-Newton matrix and the two triangular solves, as persistent kernels
// that walk a tile task graph.
//
// The matrix (row-major, edge padded to a multiple of 64 with an identity
// block) is cut into 64x64 tiles.  Right-looking blocked Cholesky as tasks:
//   POTRF(j)      L_jj = chol(A_jj), and Linv_jj = L_jj^-1        (one CTA)
//   TRSM(i,j)     L_ij = A_ij Linv_jj^T                      i > j
//   UPDATE(i,k,j) A_ik -= L_ij L_kj^T                        i >= k > j
// and for the solves
//   FWD(i)        y_i = Linv_ii (b_i - sum_{j<i} L_ij y_j)
//   BWD(i)        x_i = Linv_ii^T (y_i - sum_{j>i} L_ji^T x_j)
// CTAs take tasks in list order (one atomic counter; the list is decoded,
// not stored) and wait, with a bounded spin, for the counters of the tiles
// they read.  Every dependency of a task lies earlier in the list, so the
// earliest unfinished task can always run and the graph cannot deadlock; the
// list puts the next panel's POTRF/TRSM right after the updates they need
// (look-ahead of one panel), and one CTA (the walker) runs the diagonal
// chain POTRF -> TRSM -> UPDATE itself, so the critical path overlaps the
// bulk of the trailing updates.  The solves take their tasks the same way
// but wait on the solved blocks themselves (tagged words, below).
//
// Tiles written by one SM and read by another are moved through L2 only
// (ld.global.cg / st.global.cg) and published by a release store of the
// tile's counter, made after the block barrier that follows the stores.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <type_traits>

#include "sc_common.cuh"

namespace sc {

enum TaskType { T_POTRF = 0, T_TRSM = 1, T_UPD = 2, T_FWD = 3, T_BWD = 4 };

// sync area (ints): [0] factor task counter, [1] solve task counter (and,
// during a factorisation, the walker's SM + 1), upd[nT*nT], potrf_done[nT],
// trsm_done[nT*nT].  The solves pass their blocks as tagged words instead.
struct SyncView {
  int* fctr;
  int* sctr;
  int* upd;
  int* pdone;
  int* tdone;
  __host__ __device__ SyncView(int* s, int nT)
      : fctr(s), sctr(s + 1), upd(s + 2), pdone(s + 2 + nT * nT), tdone(s + 2 + nT * nT + nT) {}
};

int chol_sync_ints(int nT) { return 2 + 2 * nT * nT + nT; }
// a factorisation resets the whole sync area
static int chol_factor_reset_ints(int nT) { return chol_sync_ints(nT); }

// Task t of the factorisation list (decoded, no list in memory):
//   POTRF(0), TRSM(1..nT-1, 0), then for each panel j = 0..nT-2:
//   UPDATE(j+1..nT-1, j+1, j)   -- the next panel column first
//   POTRF(j+1), TRSM(j+2..nT-1, j+1)
//   UPDATE(i, k, j) for k = j+2..nT-1, i = k..nT-1
// Returned as (type, i, k, j); type -1 past the end.
// Tasks in the panel blocks whose size parameter m (= nT - 1 - j) runs from
// 1 to x: block j holds m + 1 + (m - 1) + (m - 1) m / 2 = (m^2 + 3m) / 2
// tasks, and the sum of (m^2 + 3m) / 2 over m = 1..x is x (x+1) (x+5) / 6.
__host__ __device__ __forceinline__ long long chol_panel_tasks(long long x) { return x * (x + 1) * (x + 5) / 6; }

// Decodes list position t in O(1): the panel block from a cube-root estimate
// of the inverse of chol_panel_tasks, the trailing-update column from the
// quadratic formula, each estimate corrected by exact integer comparisons.
__host__ __device__ int4 chol_task(int nT, int t) {
  if (t == 0) return make_int4(T_POTRF, 0, 0, 0);
  if (t < nT) return make_int4(T_TRSM, t, 0, 0);
  const long long r = (long long)t - nT;  // rank among the panel blocks
  const long long total = chol_panel_tasks(nT - 1);
  if (r >= total) return make_int4(-1, 0, 0, 0);
  // block with the smallest m such that the blocks m..1 hold >= total - r tasks
  const long long left = total - r;
  int m = (int)cbrtf(6.0f * (float)left);
  if (m < 1) m = 1;
  if (m > nT - 1) m = nT - 1;
  while (chol_panel_tasks(m) < left) ++m;
  while (m > 1 && chol_panel_tasks(m - 1) >= left) --m;
  const int j = nT - 1 - m, m2 = m - 1;
  int rel = (int)(r - (total - chol_panel_tasks(m)));
  if (rel < m) return make_int4(T_UPD, j + 1 + rel, j + 1, j);
  rel -= m;
  if (rel == 0) return make_int4(T_POTRF, j + 1, j + 1, j + 1);
  rel -= 1;
  if (rel < m2) return make_int4(T_TRSM, j + 2 + rel, j + 1, j + 1);
  rel -= m2;
  // trailing columns k = j+2.. hold m2, m2-1, ... tasks; column n starts at
  // n m2 - n (n-1) / 2
  const float bq = 2.0f * m2 + 1.0f;
  int n = (int)((bq - sqrtf(fmaxf(bq * bq - 8.0f * rel, 0.0f))) * 0.5f);
  if (n < 0) n = 0;
  auto start = [m2](int c) { return c * m2 - c * (c - 1) / 2; };
  while (n > 0 && start(n) > rel) --n;
  while (n + 1 < m2 && start(n + 1) <= rel) ++n;
  const int k = j + 2 + n;
  return make_int4(T_UPD, k + (rel - start(n)), k, j);
}

int chol_ntasks(int nT) { return nT + (int)chol_panel_tasks(nT - 1); }

// Solve list: FWD(0..nT-1), then BWD(nT-1..0).
__host__ __device__ int4 solve_task(int nT, int t) {
  if (t < nT) return make_int4(T_FWD, t, 0, 0);
  if (t < 2 * nT) return make_int4(T_BWD, 2 * nT - 1 - t, 0, 0);
  return make_int4(-1, 0, 0, 0);
}

// ---- synchronisation primitives -----------------------------------------------------------

constexpr long kSpinLimit = 1L << 22;  // ~1 s of polling with the back-off below

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Publishes a counter.  Callers reach it through a __syncthreads() after
// the block's stores of the tile; a release store is cumulative, so those
// stores of every thread of the block become visible before the counter.
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_status(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Waits until *p >= v (the counters only grow).  The first read is an
// acquire load, which settles the common case of a dependency finished long
// ago in one round trip.  Otherwise it polls with relaxed loads (an acquire
// load on every poll would invalidate this SM's L1 each time and stall the
// load/store path of the other CTAs sharing the SM) and confirms with one
// acquire load once the value is seen.  An acquire load, unlike a fence,
// does not wait for this thread's earlier stores and atomics to complete.
// Gives up (returns false) after kSpinLimit polls or as soon as another
// CTA has recorded a timeout.
__device__ bool wait_ge(const int* p, int v, uint32_t* status) {
  if (ld_acquire(p) >= v) return true;
  for (long it = 0; it < kSpinLimit; ++it) {
    __nanosleep(it < 16 ? 32 : 200);
    if (ld_relaxed(p) >= v) return ld_acquire(p) >= v;
    if ((it & 63) == 63 && (ld_status(status) & SC_STATUS_TIMEOUT)) return false;
  }
  atomicOr(status, SC_STATUS_TIMEOUT);
  return false;
}

// ---- tile helpers --------------------------------------------------------------------------

// Shared-memory row pitch: 64 elements + 16 bytes, so that rows stay 16-byte
// aligned for vector loads and consecutive rows start 4 banks apart.
template <typename R>
struct Pitch {
  static constexpr int value = kNB + 16 / (int)sizeof(R);
};

// 64x64 tile moves between global memory (through L2 only) and shared
// memory in 16-byte vectors: each thread issues 4 (float) or 8 (double)
// independent requests instead of 16.
template <typename R>
__device__ __forceinline__ void load_tile(R* sm, const R* g, int lda) {
  constexpr int LD = Pitch<R>::value;
  constexpr int V = 16 / (int)sizeof(R);  // elements per vector
  constexpr int PER_ROW = kNB / V;
  for (int e = threadIdx.x; e < kNB * PER_ROW; e += blockDim.x) {
    int r = e / PER_ROW, c = (e - r * PER_ROW) * V;
    float4 v = __ldcg(reinterpret_cast<const float4*>(g + (size_t)r * lda + c));
    *reinterpret_cast<float4*>(sm + r * LD + c) = v;
  }
}
// The same copy issued as 16-byte cp.async requests (L2 only); the caller
// commits the group.
template <typename R>
__device__ __forceinline__ void copy_tile_async(R* sm, const R* g, int lda) {
  constexpr int LD = Pitch<R>::value;
  constexpr int PER_ROW = kNB * (int)sizeof(R) / 16;
  for (int e = threadIdx.x; e < kNB * PER_ROW; e += blockDim.x) {
    int r = e / PER_ROW, ch = e - r * PER_ROW;
    const char* src = reinterpret_cast<const char*>(g + (size_t)r * lda) + 16 * ch;
    unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<char*>(sm + r * LD) + 16 * ch);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
  }
}
__device__ __forceinline__ void async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void async_wait_prev() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

template <typename R>
__device__ __forceinline__ void store_tile(R* g, int lda, const R* sm) {
  constexpr int LD = Pitch<R>::value;
  constexpr int V = 16 / (int)sizeof(R);
  constexpr int PER_ROW = kNB / V;
  for (int e = threadIdx.x; e < kNB * PER_ROW; e += blockDim.x) {
    int r = e / PER_ROW, c = (e - r * PER_ROW) * V;
    __stcg(reinterpret_cast<float4*>(g + (size_t)r * lda + c), *reinterpret_cast<const float4*>(sm + r * LD + c));
  }
}

// acc[a][b] = sum_m X[ty+16a][m] Y[tx+16b][m]   (X Y^T on 64x64 tiles); the
// contraction index is contiguous in both operands, so each thread reads
// 16-byte vectors along it.
__device__ __forceinline__ void gemm_nt(float acc[4][4], const float* X, const float* Y) {
  constexpr int L = Pitch<float>::value;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll
  for (int m = 0; m < kNB; m += 4) {
    float4 x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = *reinterpret_cast<const float4*>(X + (ty + 16 * a) * L + m);
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = *reinterpret_cast<const float4*>(Y + (tx + 16 * b) * L + m);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        float t = acc[a][b];
        t = fmaf(x[a].x, y[b].x, t);
        t = fmaf(x[a].y, y[b].y, t);
        t = fmaf(x[a].z, y[b].z, t);
        t = fmaf(x[a].w, y[b].w, t);
        acc[a][b] = t;
      }
  }
}
__device__ __forceinline__ void gemm_nt(double acc[4][4], const double* X, const double* Y) {
  constexpr int L = Pitch<double>::value;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
#pragma unroll 2
  for (int m = 0; m < kNB; m += 2) {
    double2 x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = *reinterpret_cast<const double2*>(X + (ty + 16 * a) * L + m);
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = *reinterpret_cast<const double2*>(Y + (tx + 16 * b) * L + m);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a].y, y[b].y, fma(x[a].x, y[b].x, acc[a][b]));
  }
}

// Reciprocal of an elimination pivot: the hardware approximation (relative
// error below 2^-22) in float32, the rounded reciprocal in float64.
__device__ __forceinline__ float pivot_rcp(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ double pivot_rcp(double x) { return __drcp_rn(x); }

// Compile-time loops: every step below is instantiated with constant
// indices, so the per-lane rows stay in registers.
template <int I, int N>
struct Static {
  template <typename F>
  __device__ __forceinline__ static void each(F&& f) {
    f(std::integral_constant<int, I>());
    Static<I + 1, N>::each(f);
  }
};
template <int N>
struct Static<N, N> {
  template <typename F>
  __device__ __forceinline__ static void each(F&&) {}
};

// gemm_nt restricted to the terms that can be nonzero, for the walker's
// chain products:
//   TRI_Y: Y is lower triangular (Y[c][m] = 0 for m > c, as Linv_jj is
//          stored), so output column block b sums only m < 16 (b + 1);
//   SYM:   X Y^T is symmetric and only its lower part is read, so only the
//          16x16 blocks a >= b are formed (the others are left unset).
// The skipped terms are exact zeros, and the kept ones are added in gemm_nt's
// order, so every formed entry has gemm_nt's value.
template <bool TRI_Y, bool SYM>
__device__ __forceinline__ void gemm_nt_part(float acc[4][4], const float* X, const float* Y) {
  constexpr int L = Pitch<float>::value;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  Static<0, 4>::each([&](auto mc_) {  // contraction chunk m = 16 mc .. 16 mc + 15
    constexpr int mc = decltype(mc_)::value;
#pragma unroll
    for (int m = 16 * mc; m < 16 * mc + 16; m += 4) {
      float4 x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = *reinterpret_cast<const float4*>(X + (ty + 16 * a) * L + m);
      Static<0, 4>::each([&](auto b_) {
        constexpr int b = decltype(b_)::value;
        if constexpr (!TRI_Y || b >= mc) y[b] = *reinterpret_cast<const float4*>(Y + (tx + 16 * b) * L + m);
      });
      Static<0, 4>::each([&](auto a_) {
        constexpr int a = decltype(a_)::value;
        Static<0, 4>::each([&](auto b_) {
          constexpr int b = decltype(b_)::value;
          if constexpr ((!TRI_Y || b >= mc) && (!SYM || a >= b)) {
            float t = acc[a][b];
            t = fmaf(x[a].x, y[b].x, t);
            t = fmaf(x[a].y, y[b].y, t);
            t = fmaf(x[a].z, y[b].z, t);
            t = fmaf(x[a].w, y[b].w, t);
            acc[a][b] = t;
          }
        });
      });
    }
  });
}
template <bool TRI_Y, bool SYM>
__device__ __forceinline__ void gemm_nt_part(double acc[4][4], const double* X, const double* Y) {
  constexpr int L = Pitch<double>::value;
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
  Static<0, 4>::each([&](auto mc_) {
    constexpr int mc = decltype(mc_)::value;
#pragma unroll 2
    for (int m = 16 * mc; m < 16 * mc + 16; m += 2) {
      double2 x[4], y[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) x[a] = *reinterpret_cast<const double2*>(X + (ty + 16 * a) * L + m);
      Static<0, 4>::each([&](auto b_) {
        constexpr int b = decltype(b_)::value;
        if constexpr (!TRI_Y || b >= mc) y[b] = *reinterpret_cast<const double2*>(Y + (tx + 16 * b) * L + m);
      });
      Static<0, 4>::each([&](auto a_) {
        constexpr int a = decltype(a_)::value;
        Static<0, 4>::each([&](auto b_) {
          constexpr int b = decltype(b_)::value;
          if constexpr ((!TRI_Y || b >= mc) && (!SYM || a >= b))
            acc[a][b] = fma(x[a].y, y[b].y, fma(x[a].x, y[b].x, acc[a][b]));
        });
      });
    }
  });
}

// 16 consecutive values at a 16-byte aligned shared-memory address.
__device__ __forceinline__ void ld16(const float* p, float (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    float4 t = reinterpret_cast<const float4*>(p)[u];
    v[4 * u] = t.x;
    v[4 * u + 1] = t.y;
    v[4 * u + 2] = t.z;
    v[4 * u + 3] = t.w;
  }
}
__device__ __forceinline__ void ld16(const double* p, double (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    double2 t = reinterpret_cast<const double2*>(p)[u];
    v[2 * u] = t.x;
    v[2 * u + 1] = t.y;
  }
}
__device__ __forceinline__ void st16(float* p, const float (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 4; ++u)
    reinterpret_cast<float4*>(p)[u] = make_float4(v[4 * u], v[4 * u + 1], v[4 * u + 2], v[4 * u + 3]);
}
__device__ __forceinline__ void st16(double* p, const double (&v)[16]) {
#pragma unroll
  for (int u = 0; u < 8; ++u) reinterpret_cast<double2*>(p)[u] = make_double2(v[2 * u], v[2 * u + 1]);
}

// In-place Cholesky of the 64x64 SPD tile in sm (pitch of the tile, lower
// part read), writing L (upper part zeroed) to sm and L^-1 to sv
// (potrf_tile_w below).
//
// Gaussian elimination in LDL^T form over the rows of [A | Y], Y = I at the
// start, W columns per step.  With A = L' D L'^T (L' unit lower,
// D = diag(p)), L = L' D^1/2 and L^-1 = D^-1/2 L'^-1; the elimination turns
// Y into L'^-1.  Step k eliminates columns K = k..k+W-1 at once: with
// V = A[:, K] and Z = Y[K, :] as they stand before the step, and the W x W
// pivot block V[K, :] = L_D P L_D^T factorised by every thread, row i gets
//   u_i = V[i, :] L_D^-T          (A[i][k+m] at step k+m: final for column k+m)
//   g_i[m] = u_i[m] / p_m         (zero unless i > k+m)
//   c_i = g_i L_D^-1
//   A[i][j] -= c_i . V[j, :]      (j > k+W-1)
//   Y[i][:] -= c_i . Z            (equals the W single-column steps)
// Afterwards L[i][j] = A[i][j] / sqrt(p_j) for j < i, L[j][j] = sqrt(p_j),
// (L^-1)[i][c] = Y[i][c] / sqrt(p_i).  A non-positive pivot is replaced by
// 1 and sets *bad.
//
// Thread layout: warp w owns column block q = w % 4 (columns 16q..16q+15)
// of rows 32 (w / 4) .. +31, one row per lane, 16 entries of A and 16 of Y
// in registers.  Each step reads the published columns K of A and rows K of
// Y from shared memory (double-buffered, one barrier per step); the owners
// of the next W columns and rows publish them.  Once k >= 32 the rows 0..31
// are final (their multipliers c are zero), so their warps skip the row
// work and only take part in the pivots and the barriers; warp w runs on
// scheduler w % 4 of the SM, so each scheduler keeps one working warp.
template <typename R>
__device__ __forceinline__ R pivot_guard(R p, int* bad) {
  if (!(p > (R)0)) {
    if (threadIdx.x == 0) *bad = 1;
    return (R)1;
  }
  return p;
}

// Columns per elimination step of potrf_tile.  8 halves the steps (and
// barriers) of 4, each a longer chain of pivots; measured at order 4096 on
// GB300 it was no faster (1237 against 1233 us per factorisation), so 4.
#ifndef SC_POTRF_W
#define SC_POTRF_W 4
#endif

// The elimination above, W columns per step (W = 4 or 8).  The pivot
// block V[K, :] (W x W) is factorised by every thread in LDL^T form by
// right-looking elimination; a row's u, g and c follow the formulas above
// with W terms; the updates add the W rank-one terms in column order.
// aux: [2][W][64] published columns, [2][W][64] published rows of Y, [64]
// pivots (4 W 64 + 64 values).
template <int W, typename R>
__device__ void potrf_tile_w(R* sm, R* sv, R* aux, int* bad) {
  static_assert(W == 4 || W == 8, "4 or 8 columns per step");
  constexpr int LD = Pitch<R>::value;
  constexpr int S = 16 / W;  // steps per 16-column block
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = warp & 3, h = warp >> 2, i = 32 * h + lane, cb = 16 * q;
  R* colb = aux;               // [2][W][64]: colb[m][j] = A[j][k+m]
  R* rowb = aux + 2 * W * 64;  // [2][W][64]: rowb[m][c] = Y[k+m][c]
  R* piv = aux + 4 * W * 64;   // [64] pivots
  R a[16], y[16];
  ld16(sm + i * LD + cb, a);
  Static<0, 16>::each([&](auto tt) {
    constexpr int t = decltype(tt)::value;
    y[t] = (cb + t == i) ? (R)1 : (R)0;
  });
  if (q == 0) {
#pragma unroll
    for (int m = 0; m < W; ++m) colb[64 * m + i] = a[m];
  }
  if (i < W) st16(rowb + 64 * i + cb, y);
  __syncthreads();
  for (int kb = 0; kb < 4; ++kb) {
    Static<0, S>::each([&](auto kq_) {
      constexpr int kq = decltype(kq_)::value;
      constexpr int bsel = kq & 1;  // parity of the step index S kb + kq (S = 2 or 4, so S kb is even)
      constexpr int t0 = W * kq;    // first column of K inside block q == kb
      const int k = 16 * kb + t0;
      const R* col = colb + W * 64 * bsel;
      const R* row = rowb + W * 64 * bsel;
      R* coln = colb + W * 64 * (bsel ^ 1);
      R* rown = rowb + W * 64 * (bsel ^ 1);
      // pivot block E = V[K, :] (lower part), eliminated in place: L, p
      R E[W][W], L[W][W], p[W], r[W];
#pragma unroll
      for (int m = 0; m < W; ++m)
#pragma unroll
        for (int n = 0; n <= m; ++n) E[m][n] = col[64 * n + k + m];
#pragma unroll
      for (int n = 0; n < W; ++n) {
        p[n] = pivot_guard(E[n][n], bad);
        r[n] = pivot_rcp(p[n]);
#pragma unroll
        for (int m = n + 1; m < W; ++m) L[m][n] = E[m][n] * r[n];
#pragma unroll
        for (int m = n + 1; m < W; ++m)
#pragma unroll
          for (int o = n + 1; o <= m; ++o) E[m][o] = fma(-L[m][n], E[o][n], E[m][o]);
      }
      if (threadIdx.x == 0) {
#pragma unroll
        for (int m = 0; m < W; ++m) piv[k + m] = p[m];
      }
      // every row of this warp is at most k: c = 0, the row work is a no-op
      if (32 * h + 31 <= k) {
        __syncthreads();
        return;
      }
      // this row: u = V[i,:] L_D^-T, g = masked u / p, c = g L_D^-1
      R u[W], c[W];
#pragma unroll
      for (int m = 0; m < W; ++m) {
        u[m] = col[64 * m + i];
#pragma unroll
        for (int n = 0; n < m; ++n) u[m] = fma(-L[m][n], u[n], u[m]);
      }
#pragma unroll
      for (int m = W - 1; m >= 0; --m) {
        c[m] = i > k + m ? u[m] * r[m] : (R)0;
#pragma unroll
        for (int n = m + 1; n < W; ++n) c[m] = fma(-c[n], L[n][m], c[m]);
      }
      // A[i][j] -= c . V[j,:] for the columns j > k+W-1 of this block
      if (q >= kb) {
        if (q == kb) {
#pragma unroll
          for (int m = 0; m < W; ++m) a[t0 + m] = u[m];
        }
#pragma unroll
        for (int m = 0; m < W; ++m) {
          R v[16];
          ld16(col + 64 * m + cb, v);
          if (q > kb) {
            Static<0, 16>::each([&](auto tt) {
              constexpr int t = decltype(tt)::value;
              a[t] = fma(-c[m], v[t], a[t]);
            });
          } else {
            Static<t0 + W, 16>::each([&](auto tt) {
              constexpr int t = decltype(tt)::value;
              a[t] = fma(-c[m], v[t], a[t]);
            });
          }
        }
      }
      // Y[i][:] -= c . W; W[m][col] is zero right of column k+m
      if (q <= kb) {
#pragma unroll
        for (int m = 0; m < W; ++m) {
          R w[16];
          ld16(row + 64 * m + cb, w);
          Static<0, 16>::each([&](auto tt) {
            constexpr int t = decltype(tt)::value;
            y[t] = fma(-c[m], w[t], y[t]);
          });
        }
      }
      // publish the next W columns of A and rows of Y
      if (k + W < 64) {
        if constexpr (kq < S - 1) {
          if (q == kb) {
#pragma unroll
            for (int m = 0; m < W; ++m) coln[64 * m + i] = a[t0 + W + m];
          }
        } else {
          if (q == kb + 1) {
#pragma unroll
            for (int m = 0; m < W; ++m) coln[64 * m + i] = a[m];
          }
        }
        if (i >= k + W && i < k + 2 * W) st16(rown + 64 * (i - k - W) + cb, y);
      }
      __syncthreads();
    });
  }
  R pj[16];
  ld16(piv + cb, pj);
  const R ri = rsqrt(piv[i]);
  Static<0, 16>::each([&](auto tt) {
    constexpr int t = decltype(tt)::value;
    const int j = cb + t;
    const R rj = rsqrt(pj[t]);
    a[t] = j < i ? a[t] * rj : (j == i ? pj[t] * rj : (R)0);
    y[t] = j <= i ? y[t] * ri : (R)0;
  });
  st16(sm + i * LD + cb, a);
  st16(sv + i * LD + cb, y);
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ void potrf_tile(R* sm, R* sv, R* aux, int* bad) {
  potrf_tile_w<SC_POTRF_W>(sm, sv, aux, bad);
}

// ---- tensor-core tile products (tcgen05, 3xTF32) ---------------------------------------
//
// In float32 the TRSM and UPDATE tiles of the bulk run on the tensor cores.
// Both products are "NT" (C = X Y^T with X and Y row-major 64x64 tiles, so
// both operands are K-major): X = A_ij, Y = Linv_jj for TRSM(i, j); X = L_ij,
// Y = L_kj for UPDATE(i, k, j).  One thread issues two 2-D TMA loads per
// operand (boxes of 64 rows x 32 floats with the 128-byte swizzle, which is
// the tensor cores' K-major SW128 layout), completing on an mbarrier.  The
// block then splits every operand x into x_hi = tf32(x) and x_lo = tf32(x -
// x_hi) in place, and one thread issues, per step of K = 8, the three
// products X_lo Y_hi, X_hi Y_lo and X_hi Y_hi (the 3xTF32 scheme, about
// 2^-21 relative error per product against 2^-24 in float32) into a float32
// accumulator in tensor memory, then commits to a second mbarrier.  The
// instruction shape is M = 128, N = 64: the tile fills rows 0..63 and rows
// 64..127 read the next 8 KB of the operand region, whose results are
// never read.  Four warps read the accumulator back (tcgen05.ld, one row of
// 32 columns per thread) and store C (TRSM) or the old tile minus C
// (UPDATE).  Every mbarrier wait is bounded; a wait that gives up records
// SC_STATUS_TIMEOUT, and the block still frees its tensor memory.
namespace tc {

__device__ __forceinline__ uint32_t saddr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier (every thread of the block
// calls it); false after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (mbar_test(bar, parity)) return true;
    if (it >= 8) __nanosleep(64);
  }
  return false;
}

__device__ __forceinline__ void tma_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          saddr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(saddr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// whole warp
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(slot)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Shared-memory descriptor of a K-major operand in the 128-byte-swizzled
// layout: 8-row groups of 128-byte rows 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t addr) {
  uint64_t d = (uint64_t)((addr & 0x3FFFFu) >> 4);  // start address
  d |= (uint64_t)1 << 16;                           // leading byte offset (unused by this layout)
  d |= (uint64_t)(1024 >> 4) << 32;                 // stride byte offset
  d |= (uint64_t)1 << 46;                           // descriptor version
  d |= (uint64_t)2 << 61;                           // 128-byte swizzle
  return d;
}
// kind::tf32, float32 accumulator, both operands K-major, M = 128, N = 64
constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t accum) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(kIdesc), "r"(accum));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar))
               : "memory");
}

// 32 consecutive float32 columns of one accumulator row per thread (the
// warp's lane quadrant), then the wait for the load
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x rounded to TF32 (10 explicit mantissa bits), to nearest with ties away
// from zero, by integer operations on the bit pattern (the conversion
// instruction is several times slower); exact for the finite values of a
// positive definite factorisation, which are far from overflow.
__device__ __forceinline__ float tf32_hi(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// Splits the 64x64 tile at hi (16 KB, any layout) into hi = tf32(x) in place
// and lo = x - hi (exact; the tensor core reads its top 19 bits) at lo; the
// 256 threads take 16-byte vectors.  |x - hi - tf32(lo)| < 2^-21 |x|.
__device__ __forceinline__ void split_tile(float* hi, float* lo) {
  float4* h = reinterpret_cast<float4*>(hi);
  float4* l = reinterpret_cast<float4*>(lo);
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = threadIdx.x + 256 * u;
    const float4 x = h[e];
    const float4 a = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
    h[e] = a;
    l[e] = make_float4(x.x - a.x, x.y - a.y, x.z - a.z, x.w - a.w);
  }
}

// Operand region: X hi, X lo, Y hi, Y lo, each a 64x64 tile as two K blocks
// (columns 0..31, 32..63) of 64 rows x 128 bytes.  The M = 128 instruction
// reads 128 rows of X, so every X block is followed by 8 KB of the region.
constexpr uint32_t kTile = 64 * 64 * 4;  // 16 KB
constexpr uint32_t kKBlk = 64 * 128;      // 8 KB
constexpr uint32_t kTmemCols = 64;

}  // namespace tc

// ---- factorisation ---------------------------------------------------------------------------

// Tasks of the diagonal chain, run by one CTA (the "walker") without flag
// round trips: POTRF(j), TRSM(j+1, j), UPDATE(j+1, j+1, j) for every j.
__device__ __forceinline__ bool walker_task(int4 tk) {
  return tk.x == T_POTRF || (tk.x == T_TRSM && tk.y == tk.w + 1) ||
         (tk.x == T_UPD && tk.y == tk.w + 1 && tk.z == tk.w + 1);
}

// The walker: keeps the diagonal tile, its inverse and the next panel tile
// in shared memory and walks the critical path of the factorisation,
// publishing each result for the other CTAs.  Its own tasks appear in the
// list in the order it runs them, and it waits only on earlier tasks, so the
// list-order argument against deadlock still holds.  TRSM(j+1, j) skips the
// zero upper part of Linv_jj, and UPDATE(j+1, j+1, j) forms only the lower
// blocks that POTRF(j+1) reads; both give the sums of the full products.
template <typename R>
__device__ __noinline__ void chol_walker(R* A, int lda, int nT, R* Linv, SyncView& sv, uint32_t* status, LMState* lm,
                            R* T0, R* T1, R* T2, R* aux, int* s_bad, int* s_ok) {
  constexpr int LD = Pitch<R>::value;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  load_tile(T0, A, lda);
  for (int j = 0; j < nT; ++j) {
    if (threadIdx.x == 0) *s_bad = 0;
    __syncthreads();
    R* Ajj = A + (size_t)j * kNB * lda + (size_t)j * kNB;
    potrf_tile(T0, T1, aux, s_bad);                 // T0 = L_jj, T1 = Linv_jj
    store_tile(Ajj, lda, T0);
    store_tile(Linv + (size_t)j * kNB * kNB, kNB, T1);
    __syncthreads();
    if (threadIdx.x == 0) {
      if (*s_bad) {
        atomicOr(status, SC_STATUS_NOTPD);
        if (lm != nullptr) lm->notpd = 1;
      }
      st_release(sv.pdone + j, 1);
    }
    if (j + 1 == nT) break;
    // TRSM(j+1, j): L_{j+1,j} = A_{j+1,j} Linv_jj^T, kept in T2
    R* Ap = A + (size_t)(j + 1) * kNB * lda + (size_t)j * kNB;
    if (threadIdx.x == 0) *s_ok = wait_ge(sv.upd + (j + 1) * nT + j, j, status);
    __syncthreads();
    if (!*s_ok) {
      if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
      return;
    }
    load_tile(T2, Ap, lda);
    __syncthreads();
    R acc[4][4];
    gemm_nt_part<true, false>(acc, T2, T1);
    __syncthreads();
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int r = ty + 16 * a, c = tx + 16 * b;
        T2[r * LD + c] = acc[a][b];
        __stcg(Ap + (size_t)r * lda + c, acc[a][b]);
      }
    __syncthreads();
    if (threadIdx.x == 0) {
      st_release(sv.tdone + (j + 1) * nT + j, 1);
    }
    // UPDATE(j+1, j+1, j): the next diagonal tile, kept in T0 for POTRF(j+1)
    if (threadIdx.x == 0) *s_ok = wait_ge(sv.upd + (j + 1) * nT + (j + 1), j, status);
    __syncthreads();
    if (!*s_ok) {
      if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
      return;
    }
    load_tile(T0, A + (size_t)(j + 1) * kNB * lda + (size_t)(j + 1) * kNB, lda);
    __syncthreads();
    gemm_nt_part<false, true>(acc, T2, T2);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b <= a; ++b) T0[(ty + 16 * a) * LD + tx + 16 * b] -= acc[a][b];
  }
}

// Dependency counter q (0..2) of a TRSM or UPDATE task and the value it
// must reach; p = nullptr where the task has fewer counters.
__device__ __forceinline__ void task_dep(int4 tk, int nT, const SyncView& sv, int q, const int*& p, int& v) {
  const int i = tk.y, k = tk.z, j = tk.w;
  p = nullptr;
  v = 0;
  if (tk.x == T_TRSM) {
    if (q == 0) p = sv.pdone + j, v = 1;
    else if (q == 1) p = sv.upd + i * nT + j, v = j;
  } else {
    if (q == 0) p = sv.tdone + i * nT + j, v = 1;
    else if (q == 1) p = sv.tdone + k * nT + j, v = 1;
    else p = sv.upd + i * nT + k, v = j;
  }
}

// Queues the operand tiles of a TRSM (A_ij, Linv_jj) or UPDATE (L_ij, L_kj)
// task into X and Y as one cp.async group.
template <typename R>
__device__ __forceinline__ void task_operands_async(int4 tk, const R* A, int lda, const R* Linv, R* X, R* Y) {
  const int i = tk.y, k = tk.z, j = tk.w;
  copy_tile_async(X, A + (size_t)i * kNB * lda + (size_t)j * kNB, lda);
  if (tk.x == T_TRSM) copy_tile_async(Y, Linv + (size_t)j * kNB * kNB, kNB);
  else copy_tile_async(Y, A + (size_t)k * kNB * lda + (size_t)j * kNB, lda);
  async_commit();
}

// Queues the operand tiles of a TRSM (A_ij, Linv_jj) into X and Y, or of an
// UPDATE (L_ij, L_kj) into X and Y with its output tile A_ik into O, as one
// cp.async group: the block then holds no copy of the output in registers.
template <typename R>
__device__ __forceinline__ void task_tiles_async(int4 tk, const R* A, int lda, const R* Linv, R* X, R* Y, R* O) {
  const int i = tk.y, k = tk.z, j = tk.w;
  copy_tile_async(X, A + (size_t)i * kNB * lda + (size_t)j * kNB, lda);
  if (tk.x == T_TRSM) {
    copy_tile_async(Y, Linv + (size_t)j * kNB * kNB, kNB);
  } else {
    copy_tile_async(Y, A + (size_t)k * kNB * lda + (size_t)j * kNB, lda);
    copy_tile_async(O, A + (size_t)i * kNB * lda + (size_t)k * kNB, lda);
  }
  async_commit();
}

// Persistent tile-DAG factorisation.  The block that claims task 0 becomes
// the walker.  Every other block runs TRSM and UPDATE tasks in
// list order, two deep: while it multiplies the current task, the operands
// of the task it claimed next are already on their way into the other
// buffer pair, provided that task's dependencies were complete when it
// looked (a non-blocking check); otherwise it finishes the current task
// first and then waits.  The lowest unfinished claimed task is always some
// block's current task, whose dependencies precede it in the list, so list
// order rules out deadlock.
template <typename R>
__global__ void __launch_bounds__(kCholThreads) k_chol(R* __restrict__ A, int lda, int nT,
                                                      R* __restrict__ Linv, int n_tasks,
                                                      int* sync, uint32_t* status, LMState* lm) {
  if (lm != nullptr && lm->done) return;
  constexpr int LD = Pitch<R>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* s0 = reinterpret_cast<R*>(smraw);
  R* s1 = s0 + kNB * LD;
  R* s2 = s1 + kNB * LD;
  R* aux = s2 + kNB * LD;  // the walker's scratch; the second Y buffer otherwise
  auto Xb = [&](int b) { return b ? s2 : s0; };  // buffer pairs (s0, s1) and (s2, aux)
  auto Yb = [&](int b) { return b ? aux : s1; };
  __shared__ int s_task, s_ok, s_bad;
  __shared__ int4 s_tk;  // the task at s_task, decoded once by thread 0
  SyncView sv(sync, nT);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int next = -1;  // thread 0: the claimed, not yet examined task
  // The walker publishes its SM (+1) in the otherwise idle solve counter; a
  // block sharing that SM stops claiming, finishes what it holds and
  // leaves the SM to the critical path.  A hint only: nothing depends on it.
  int walker_sm = -1, my_sm = 0;
  if (threadIdx.x == 0) asm volatile("mov.u32 %0, %%smid;" : "=r"(my_sm));
  auto claim = [&]() -> int {  // thread 0
    if (walker_sm < 0) {
      const int w = ld_relaxed(sv.sctr);
      if (w > 0) walker_sm = w - 1;
    }
    return walker_sm == my_sm ? n_tasks : atomicAdd(sv.fctr, 1);
  };
  int4 cur = make_int4(-1, 0, 0, 0);
  bool have = false;  // cur's operands are queued in buffer pair buf
  int buf = 0;
  for (;;) {
    if (!have) {
      // claim tasks until one is ours, then wait for its dependencies
      __syncthreads();  // every thread has read the previous s_task
      if (threadIdx.x == 0) {
        s_task = next >= 0 ? next : claim();
        next = -1;
        s_tk = chol_task(nT, s_task);
      }
      __syncthreads();
      const int t = s_task;
      if (t >= n_tasks) break;
      if (t == 0) {
        if (threadIdx.x == 0) st_release(sv.sctr, my_sm + 1);
        chol_walker(A, lda, nT, Linv, sv, status, lm, s0, s1, s2, aux, &s_bad, &s_ok);
        break;
      }
      cur = s_tk;
      if (walker_task(cur)) continue;
      if (threadIdx.x == 0) next = claim();
      bool ok = true;
      if (threadIdx.x < 3) {
        const int* p;
        int v;
        task_dep(cur, nT, sv, threadIdx.x, p, v);
        if (p != nullptr) ok = wait_ge(p, v, status);
      }
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
        break;
      }
      task_operands_async(cur, A, lda, Linv, Xb(buf), Yb(buf));
      have = true;
    }
    // look at the claimed next task; queue its operands if it is ready
    if (threadIdx.x == 0) {
      s_task = next;
      if (next >= 0) s_tk = chol_task(nT, next);
    }
    __syncthreads();
    const int t2 = s_task;
    int4 nxt = make_int4(-1, 0, 0, 0);
    bool staged = false;
    if (t2 >= 0 && t2 < n_tasks) {
      nxt = s_tk;
      if (walker_task(nxt)) {
        if (threadIdx.x == 0) next = -1;  // done by the walker: skip it
      } else {
        bool ready = true;
        if (threadIdx.x < 3) {
          const int* p;
          int v;
          task_dep(nxt, nT, sv, threadIdx.x, p, v);
          if (p != nullptr) ready = ld_acquire(p) >= v;
        }
        staged = __syncthreads_and(ready) != 0;
        if (staged) {
          if (threadIdx.x == 0) next = claim();
          task_operands_async(nxt, A, lda, Linv, Xb(buf ^ 1), Yb(buf ^ 1));
        }
      }
    }
    // the current task
    const int i = cur.y, k = cur.z, j = cur.w;
    const bool trsm = cur.x == T_TRSM;
    R* Out = A + (size_t)i * kNB * lda + (size_t)(trsm ? j : k) * kNB;
    R old[4][4];  // an UPDATE's output tile, fetched while the operands arrive
    if (!trsm) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) old[a][b] = __ldcg(Out + (size_t)(ty + 16 * a) * lda + tx + 16 * b);
    }
    if (staged) async_wait_prev();
    else async_wait_all();
    __syncthreads();
    R acc[4][4];
    gemm_nt(acc, Xb(buf), Yb(buf));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        __stcg(Out + (size_t)(ty + 16 * a) * lda + tx + 16 * b, trsm ? acc[a][b] : old[a][b] - acc[a][b]);
    __syncthreads();  // the tile is stored and buffer pair buf is free
    // published by a thread outside warp 0, whose lanes 0..2 go on polling
    if (threadIdx.x == 32) {
      if (trsm) st_release(sv.tdone + i * nT + j, 1);
      else st_release(sv.upd + i * nT + k, j + 1);
    }
    if (staged) {
      cur = nxt;
      buf ^= 1;
    } else {
      have = false;
    }
  }
  async_wait_all();
}


// Position m of the combined task list of a batch: (job, task of that job's
// list).  With an order table (k_batch_order), entry m holds job << 20 |
// task; without one, the lists are interleaved.  An entry outside the
// batch gives job -1 (no task: a table that is not a permutation leaves
// tasks undone, which the bounded waits report, instead of stray pointers).
__device__ __forceinline__ void batch_task(const uint32_t* __restrict__ order, int m, int G, int n, int& job,
                                           int& t) {
  if (order != nullptr) {
    const uint32_t e = __ldg(order + m);
    job = (int)(e >> 20);
    t = (int)(e & 0xFFFFFu);
    if (job >= G || t >= n) job = -1;
  } else {
    job = m % G;
    t = m / G;
  }
}

// The factorisations of a lock-step batch of G jobs in one persistent
// launch, taking the tasks of a combined list in which every job's tasks
// keep their own order (the order table staggers the jobs; see
// batch_order_pos).  The dependencies of a task (earlier tasks of its own
// job) therefore lie earlier in the combined list, and the list-order
// argument against deadlock carries over.
// There is no walker: the diagonal chain's tasks come from the list like
// the others, a POTRF running alone in its block (nothing queued behind
// it), and while one job's chain is waited on, the other blocks find the
// other jobs' tiles.  Each tile is formed by the same arithmetic as in
// k_chol (its walker's POTRF, TRSM and diagonal UPDATE included), so every
// job's factor is bit for bit the one k_chol gives.  The counter is job 0's;
// tiles, counters, status and LM state are the task's job's.
// POTRF(j) of one job of a batch, by the whole block: waits for the tile's
// updates, factorises it in shared memory (s0 = L_jj, s1 = Linv_jj, aux
// scratch) and publishes it.  Out of line, so that its registers do not
// weigh on the tile products of the batch kernel's main loop.  False if the
// wait gave up.
template <typename R>
__device__ __noinline__ bool batch_potrf(R* A, int lda, int nT, R* Linv, int j, const SyncView& sv,
                                         uint32_t* status, LMState* lm, R* s0, R* s1, R* aux, int* s_ok,
                                         int* s_bad) {
  if (threadIdx.x == 0) {
    *s_ok = wait_ge(sv.upd + j * nT + j, j, status);
    *s_bad = 0;
  }
  __syncthreads();
  if (!*s_ok) {
    if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
    return false;
  }
  R* Ajj = A + (size_t)j * kNB * lda + (size_t)j * kNB;
  load_tile(s0, Ajj, lda);
  __syncthreads();
  potrf_tile(s0, s1, aux, s_bad);
  store_tile(Ajj, lda, s0);
  store_tile(Linv + (size_t)j * kNB * kNB, kNB, s1);
  __syncthreads();
  if (threadIdx.x == 0) {
    if (*s_bad) {
      atomicOr(status, SC_STATUS_NOTPD);
      if (lm != nullptr) lm->notpd = 1;
    }
    st_release(sv.pdone + j, 1);
  }
  return true;
}

template <typename R>
__global__ void __launch_bounds__(kCholThreads, sizeof(R) == 4 ? 2 : 1) k_chol_batch(R* __restrict__ A0, int lda, int nT,
                                                            R* __restrict__ Linv0, int n_tasks, int G, size_t js,
                                                            const uint32_t* __restrict__ order,
                                                            int* sync0, uint32_t* status0, LMState* lm0) {
  constexpr int LD = Pitch<R>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* s0 = reinterpret_cast<R*>(smraw);
  R* s1 = s0 + kNB * LD;
  R* s2 = s1 + kNB * LD;
  R* aux = s2 + kNB * LD;  // POTRF scratch; the second Y buffer otherwise
  R* o0 = aux + kNB * LD;   // an UPDATE's output tile, per buffer pair
  R* o1 = o0 + kNB * LD;
  auto Xb = [&](int b) { return b ? s2 : s0; };
  auto Yb = [&](int b) { return b ? aux : s1; };
  auto Ob = [&](int b) { return b ? o1 : o0; };
  __shared__ int s_task, s_ok, s_bad, s_job;
  __shared__ int4 s_tk;  // the task at s_task and its job, decoded once by thread 0
  int* const counter = SyncView(sync0, nT).fctr;
  const int total = n_tasks * G;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  int next = -1;  // thread 0: the claimed, not yet examined task
  int4 cur = make_int4(-1, 0, 0, 0);
  int cjob = 0;       // cur's job
  bool have = false;  // cur's operands are queued in buffer pair buf
  int buf = 0;
  for (;;) {
    if (!have) {
      __syncthreads();  // every thread has read the previous s_task and left shared memory
      if (threadIdx.x == 0) {
        s_task = next >= 0 ? next : atomicAdd(counter, 1);
        next = -1;
        if (s_task < total) {
          int jb, tt;
          batch_task(order, s_task, G, n_tasks, jb, tt);
          s_job = jb;
          if (jb >= 0) s_tk = chol_task(nT, tt);
        }
      }
      __syncthreads();
      const int m = s_task;
      if (m >= total) break;
      const int job = s_job;
      if (job < 0) continue;
      LMState* lm = job_ptr(lm0, js, job);
      if (lm != nullptr && lm->done) continue;
      R* A = job_ptr(A0, js, job);
      R* Linv = job_ptr(Linv0, js, job);
      const SyncView sv(job_ptr(sync0, js, job), nT);
      uint32_t* status = job_ptr(status0, js, job);
      cur = s_tk;
      cjob = job;
      if (cur.x == T_POTRF) {
        if (!batch_potrf(A, lda, nT, Linv, cur.w, sv, status, lm, s0, s1, aux, &s_ok, &s_bad)) break;
        continue;
      }
      if (threadIdx.x == 0) next = atomicAdd(counter, 1);
      bool ok = true;
      if (threadIdx.x < 3) {
        const int* p;
        int v;
        task_dep(cur, nT, sv, threadIdx.x, p, v);
        if (p != nullptr) ok = wait_ge(p, v, status);
      }
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
        break;
      }
      task_tiles_async(cur, A, lda, Linv, Xb(buf), Yb(buf), Ob(buf));
      have = true;
    }
    // look at the claimed next task; queue its operands if it is a ready
    // TRSM or UPDATE (a POTRF waits for the buffers to be free)
    if (threadIdx.x == 0) {
      s_task = next;
      if (next >= 0 && next < total) {
        int jb, tt;
        batch_task(order, next, G, n_tasks, jb, tt);
        s_job = jb;
        if (jb >= 0) s_tk = chol_task(nT, tt);
      }
    }
    __syncthreads();
    const int t2 = s_task;
    int4 nxt = make_int4(-1, 0, 0, 0);
    int njob = 0;
    bool staged = false;
    if (t2 >= 0 && t2 < total) {
      njob = s_job;
      const LMState* nlm = njob < 0 ? nullptr : job_ptr(lm0, js, njob);
      if (njob < 0 || (nlm != nullptr && nlm->done)) {
        if (threadIdx.x == 0) next = -1;  // a finished job: nothing to do
      } else {
        nxt = s_tk;
        if (nxt.x != T_POTRF) {
          const SyncView nsv(job_ptr(sync0, js, njob), nT);
          bool ready = true;
          if (threadIdx.x < 3) {
            const int* p;
            int v;
            task_dep(nxt, nT, nsv, threadIdx.x, p, v);
            if (p != nullptr) ready = ld_acquire(p) >= v;
          }
          staged = __syncthreads_and(ready) != 0;
          if (staged) {
            if (threadIdx.x == 0) next = atomicAdd(counter, 1);
            task_tiles_async(nxt, job_ptr(A0, js, njob), lda, job_ptr(Linv0, js, njob), Xb(buf ^ 1), Yb(buf ^ 1),
                             Ob(buf ^ 1));
          }
        }
      }
    }
    // the current task
    R* A = job_ptr(A0, js, cjob);
    const SyncView sv(job_ptr(sync0, js, cjob), nT);
    const int i = cur.y, k = cur.z, j = cur.w;
    const bool trsm = cur.x == T_TRSM;
    R* Out = A + (size_t)i * kNB * lda + (size_t)(trsm ? j : k) * kNB;
    if (staged) async_wait_prev();
    else async_wait_all();
    __syncthreads();
    R acc[4][4];
    gemm_nt(acc, Xb(buf), Yb(buf));
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b)
        __stcg(Out + (size_t)(ty + 16 * a) * lda + tx + 16 * b,
               trsm ? acc[a][b] : Ob(buf)[(ty + 16 * a) * LD + tx + 16 * b] - acc[a][b]);
    __syncthreads();  // the tile is stored and buffer pair buf is free
    if (threadIdx.x == 32) {
      if (trsm) st_release(sv.tdone + i * nT + j, 1);
      else st_release(sv.upd + i * nT + k, j + 1);
    }
    if (staged) {
      cur = nxt;
      cjob = njob;
      buf ^= 1;
    } else {
      have = false;
    }
  }
  async_wait_all();
}

// The factorisation kernel of the float32 path: the walker as in k_chol; the
// bulk TRSM/UPDATE tasks on the tensor cores, two deep.  Shared memory holds
// two stages of raw operands (X, Y: 32 KB each) and one region for the low
// parts (32 KB).  While the product of the current task runs, the operands
// of the task claimed next are already arriving by TMA in the other stage,
// provided that task's dependencies were complete at a non-blocking check;
// otherwise the block finishes the current task and then waits for them.
// The lowest unfinished claimed task is always some block's current task,
// whose dependencies precede it in the list, so list order still rules out
// deadlock.  Two blocks per SM.
namespace tc {
constexpr uint32_t kStage = 2 * kTile;                  // X, Y raw (the high parts after the split)
constexpr uint32_t kLoOff = 2 * kStage;                 // X lo, Y lo
constexpr uint32_t kRegion = 2 * kStage + 2 * kTile;    // 96 KB
}  // namespace tc

__global__ void __launch_bounds__(kCholThreads, 2) k_chol_tc(const __grid_constant__ CUtensorMap tmA,
                                                        const __grid_constant__ CUtensorMap tmL, float* __restrict__ A,
                                                        int lda, int nT, float* __restrict__ Linv, int n_tasks,
                                                        int* sync, uint32_t* status, LMState* lm) {
  if (lm != nullptr && lm->done) return;
  extern __shared__ unsigned char smraw[];
  // 1024-byte alignment of the operand region, whatever precedes the dynamic array
  const uint32_t raw = tc::saddr(smraw);
  unsigned char* base = smraw + (((raw + 1023u) & ~1023u) - raw);
  float* Xl = reinterpret_cast<float*>(base + tc::kLoOff);
  float* Yl = reinterpret_cast<float*>(base + tc::kLoOff + tc::kTile);
  uint64_t* bar_load = reinterpret_cast<uint64_t*>(base + tc::kRegion);  // [2], one per stage
  uint64_t* bar_mma = bar_load + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_load + 3);
  int* ctl = reinterpret_cast<int*>(bar_load + 4);  // s_task, s_ok, s_bad
  __shared__ int4 s_tk;  // the task at ctl[0], decoded once by thread 0
  // the walker's tiles reuse the operand region (padded layout, 3.5 tiles)
  constexpr int LD = Pitch<float>::value;
  float* T0 = reinterpret_cast<float*>(base);
  float* T1 = T0 + kNB * LD;
  float* T2 = T1 + kNB * LD;
  float* aux = T2 + kNB * LD;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    tc::mbar_init(bar_load, 1);
    tc::mbar_init(bar_load + 1, 1);
    tc::mbar_init(bar_mma, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tc::tmem_alloc(tmem_slot, tc::kTmemCols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = *tmem_slot;
  // phase parities of the mbarriers and which of them have an operation in
  // flight (the same in every thread: every branch below is block-uniform)
  uint32_t ph_load[2] = {0, 0}, ph_mma = 0;
  bool pend_load[2] = {false, false}, pend_mma = false;
  SyncView sv(sync, nT);
  int walker_sm = -1, my_sm = 0;
  if (threadIdx.x == 0) asm volatile("mov.u32 %0, %%smid;" : "=r"(my_sm));
  auto claim = [&]() -> int {  // thread 0
    if (walker_sm < 0) {
      const int w = ld_relaxed(sv.sctr);
      if (w > 0) walker_sm = w - 1;
    }
    return walker_sm == my_sm ? n_tasks : atomicAdd(sv.fctr, 1);
  };
  // thread 0: the operands of task tk into stage stg
  auto issue = [&](int4 tk, int stg) {
    unsigned char* sb = base + stg * tc::kStage;
    // the tiles were written by other blocks through the generic proxy and
    // acquired by this block; make them visible to the copy engine's reads
    asm volatile("fence.proxy.async.global;" ::: "memory");
    tc::mbar_expect_tx(bar_load + stg, 2 * tc::kTile);
#pragma unroll
    for (int kb = 0; kb < 2; ++kb) {
      tc::tma_load(sb + kb * tc::kKBlk, &tmA, kNB * tk.w + 32 * kb, kNB * tk.y, bar_load + stg);
      if (tk.x == T_TRSM)
        tc::tma_load(sb + tc::kTile + kb * tc::kKBlk, &tmL, 32 * kb, kNB * tk.w, bar_load + stg);
      else
        tc::tma_load(sb + tc::kTile + kb * tc::kKBlk, &tmA, kNB * tk.w + 32 * kb, kNB * tk.z, bar_load + stg);
    }
  };
  // epilogue threads: warps 0, 1, 4, 5 read rows 32 (warp % 4) + lane and
  // columns 32 (warp / 4) .. + 31 of the accumulator
  const bool epi = (warp & 2) == 0;
  const int erow = 32 * (warp & 3) + lane, ecol = 32 * (warp >> 2);
  int next = -1;  // thread 0: the claimed, not yet examined task
  int4 cur = make_int4(-1, 0, 0, 0);
  bool have = false;  // cur's operands are on their way into stage stg
  int stg = 0;
  bool failed = false;
  for (;;) {
    if (!have) {
      // claim tasks until one is ours, then wait for its dependencies
      __syncthreads();  // every thread has read the previous ctl[0]
      if (threadIdx.x == 0) {
        ctl[0] = next >= 0 ? next : claim();
        next = -1;
        s_tk = chol_task(nT, ctl[0]);
      }
      __syncthreads();
      const int t = ctl[0];
      if (t >= n_tasks) break;
      if (t == 0) {
        if (threadIdx.x == 0) st_release(sv.sctr, my_sm + 1);
        chol_walker(A, lda, nT, Linv, sv, status, lm, T0, T1, T2, aux, ctl + 2, ctl + 1);
        break;
      }
      cur = s_tk;
      if (walker_task(cur)) continue;
      if (threadIdx.x == 0) next = claim();
      bool ok = true;
      if (threadIdx.x < 3) {
        const int* p;
        int v;
        task_dep(cur, nT, sv, threadIdx.x, p, v);
        if (p != nullptr) ok = wait_ge(p, v, status);
      }
      if (!__syncthreads_and(ok)) {
        if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
        break;
      }
      if (threadIdx.x == 0) issue(cur, stg);
      pend_load[stg] = true;
      have = true;
    }
    // look at the claimed next task; queue its operands if it is ready
    if (threadIdx.x == 0) {
      ctl[0] = next;
      if (next >= 0) s_tk = chol_task(nT, next);
    }
    __syncthreads();
    const int t2 = ctl[0];
    int4 nxt = make_int4(-1, 0, 0, 0);
    bool staged = false;
    if (t2 >= 0 && t2 < n_tasks) {
      nxt = s_tk;
      if (walker_task(nxt)) {
        if (threadIdx.x == 0) next = -1;  // done by the walker: skip it
      } else {
        bool ready = true;
        if (threadIdx.x < 3) {
          const int* p;
          int v;
          task_dep(nxt, nT, sv, threadIdx.x, p, v);
          if (p != nullptr) ready = ld_acquire(p) >= v;
        }
        staged = __syncthreads_and(ready) != 0;
        if (staged && threadIdx.x == 0) {
          next = claim();
          issue(nxt, stg ^ 1);
        }
        if (staged) pend_load[stg ^ 1] = true;
      }
    }
    // the current task
    const int i = cur.y, k = cur.z, j = cur.w;
    const bool trsm = cur.x == T_TRSM;
    float* Out = A + (size_t)i * kNB * lda + (size_t)(trsm ? j : k) * kNB;
    float* orow = Out + (size_t)erow * lda + ecol;
    float old[32];
    if (epi && !trsm) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float4 v = __ldcg(reinterpret_cast<const float4*>(orow) + u);
        old[4 * u] = v.x, old[4 * u + 1] = v.y, old[4 * u + 2] = v.z, old[4 * u + 3] = v.w;
      }
    }
    const bool landed = tc::mbar_wait(bar_load + stg, ph_load[stg]);
    if (!__syncthreads_and(landed)) {
      failed = true;
      break;
    }
    ph_load[stg] ^= 1;
    pend_load[stg] = false;
    float* Xh = reinterpret_cast<float*>(base + stg * tc::kStage);
    float* Yh = reinterpret_cast<float*>(base + stg * tc::kStage + tc::kTile);
    tc::split_tile(Xh, Xl);
    tc::split_tile(Yh, Yl);
    tc::fence_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      tc::fence_after();
      const uint32_t xh = tc::saddr(Xh), xl = tc::saddr(Xl), yh = tc::saddr(Yh), yl = tc::saddr(Yl);
#pragma unroll
      for (int s8 = 0; s8 < 8; ++s8) {  // K = 64 in steps of 8: block s8 / 4, 32 bytes each
        const uint32_t off = (s8 >> 2) * tc::kKBlk + (s8 & 3) * 32;
        tc::mma_tf32(tmem, tc::sw128_desc(xl + off), tc::sw128_desc(yh + off), s8 > 0 ? 1u : 0u);
        tc::mma_tf32(tmem, tc::sw128_desc(xh + off), tc::sw128_desc(yl + off), 1u);
        tc::mma_tf32(tmem, tc::sw128_desc(xh + off), tc::sw128_desc(yh + off), 1u);
      }
      tc::mma_commit(bar_mma);
    }
    pend_mma = true;
    const bool done = tc::mbar_wait(bar_mma, ph_mma);
    if (!__syncthreads_and(done)) {
      failed = true;
      break;
    }
    ph_mma ^= 1;
    pend_mma = false;
    tc::fence_after();
    if (epi) {
      float d[32];
      tc::tmem_ld32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)ecol, d);
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        float4 v;
        if (trsm) v = make_float4(d[4 * u], d[4 * u + 1], d[4 * u + 2], d[4 * u + 3]);
        else
          v = make_float4(old[4 * u] - d[4 * u], old[4 * u + 1] - d[4 * u + 1], old[4 * u + 2] - d[4 * u + 2],
                          old[4 * u + 3] - d[4 * u + 3]);
        __stcg(reinterpret_cast<float4*>(orow) + u, v);
      }
    }
    tc::fence_before();
    __syncthreads();  // the tile is stored; the accumulator, the stage and the low parts are free
    if (threadIdx.x == 32) {
      if (trsm) st_release(sv.tdone + i * nT + j, 1);
      else st_release(sv.upd + i * nT + k, j + 1);
    }
    if (staged) {
      cur = nxt;
      stg ^= 1;
    } else {
      have = false;
    }
  }
  // Leave no asynchronous work behind: a stage whose copies were issued and
  // not consumed, and the product after a wait that gave up, get a bounded
  // wait before the tensor memory is freed.
  __syncthreads();
  if (threadIdx.x == 0) {
    if (failed) atomicOr(status, SC_STATUS_TIMEOUT);
    for (int s2 = 0; s2 < 2; ++s2)
      if (pend_load[s2]) (void)tc::mbar_wait(bar_load + s2, ph_load[s2]);
    if (pend_mma) (void)tc::mbar_wait(bar_mma, ph_mma);
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, tc::kTmemCols);
}

// Dynamic shared memory of k_chol_tc: the operand region (which the walker
// reuses), the mbarriers, the tensor-memory slot and the control words, plus
// 1 KB for the alignment.
static size_t chol_tc_smem() { return tc::kRegion + 64 + 1024; }

// Tensor maps of the matrix (rows of lda floats) and of the diagonal-block
// inverses ([nT * 64] rows of 64 floats): 2-D, boxes of 64 rows x 32 floats,
// 128-byte swizzle.  cuTensorMapEncodeTiled is reached through the runtime's
// driver entry point, so the library needs no link to the driver library.
static cudaError_t encode_tile_map(CUtensorMap* map, const float* base, uint64_t cols, uint64_t rows,
                                   uint64_t row_bytes) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      fn = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }();
  if (encode == nullptr) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {cols, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {32, 64};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Blocks of the persistent factorisation kernel that fill the GPU (at most
// 4 per SM).  Computed once per precision; the function-local static makes
// the first computation thread safe for concurrent callers.
template <typename R>
static int chol_grid(const void* fn, size_t smem) {
  static const int cached = [&] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kCholThreads, smem);
    return std::max(1, sms * std::min(std::max(per, 1), 4));
  }();
  return cached;
}

// Blocks of k_chol_tc: two per SM, computed once.  The occupancy query
// reports one block per SM for a kernel that allocates tensor memory, but
// registers (112 a thread) and shared memory (97 KB) leave room for two, and
// two blocks allocate 128 of the 512 tensor-memory columns.  Blocks that do
// not find a slot start when others leave; tasks are claimed only by running
// blocks, so nothing waits on a block that has not started.
static int chol_tc_grid() {
  static const int cached = [] {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fn = reinterpret_cast<const void*>(&k_chol_tc);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)chol_tc_smem());
    // all of the unified L1 as shared memory: two blocks of ~97 KB per SM
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    return std::max(1, 2 * sms);
  }();
  return cached;
}

static cudaError_t launch_chol_tc(float* A, int lda, int nT, float* Linv, int* sync, uint32_t* status, LMState* lm,
                                  int max_ctas, cudaStream_t st) {
  const int n_tasks = chol_ntasks(nT);
  CUtensorMap tmA, tmL;
  cudaError_t e = encode_tile_map(&tmA, A, (uint64_t)lda, (uint64_t)nT * kNB, (uint64_t)lda * sizeof(float));
  if (e != cudaSuccess) return e;
  e = encode_tile_map(&tmL, Linv, kNB, (uint64_t)nT * kNB, kNB * sizeof(float));
  if (e != cudaSuccess) return e;
  int grid = std::min(chol_tc_grid(), n_tasks);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  e = cudaMemsetAsync(sync, 0, sizeof(int) * chol_factor_reset_ints(nT), st);
  if (e != cudaSuccess) return e;
  k_chol_tc<<<grid, kCholThreads, chol_tc_smem(), st>>>(tmA, tmL, A, lda, nT, Linv, n_tasks, sync, status, lm);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_chol(R* A, int lda, int nT, R* Linv, int* sync, uint32_t* status, LMState* lm,
                        int max_ctas, int kernel, cudaStream_t st) {
  if constexpr (sizeof(R) == 4) {
    if (kernel == SC_CHOL_TENSOR) return launch_chol_tc(A, lda, nT, Linv, sync, status, lm, max_ctas, st);
  }
  int n_tasks = chol_ntasks(nT);
  size_t smem = sizeof(R) * (4 * kNB) * Pitch<R>::value;  // two buffer pairs; the walker uses 3.5 tiles
  const void* fn = reinterpret_cast<const void*>(&k_chol<R>);
  int grid = std::min(chol_grid<R>(fn, smem), n_tasks);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(int) * chol_factor_reset_ints(nT), st);
  if (e != cudaSuccess) return e;
  k_chol<R><<<grid, kCholThreads, smem, st>>>(A, lda, nT, Linv, n_tasks, sync, status, lm);
  return cudaGetLastError();
}
template cudaError_t launch_chol<float>(float*, int, int, float*, int*, uint32_t*, LMState*, int, int,
                                        cudaStream_t);
template cudaError_t launch_chol<double>(double*, int, int, double*, int*, uint32_t*, LMState*, int, int,
                                         cudaStream_t);

// Blocks of k_chol_batch: as many as are resident at once, computed once.
template <typename R>
static int chol_batch_grid(size_t smem) {
  static const int cached = [&] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* fn = reinterpret_cast<const void*>(&k_chol_batch<R>);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    // all of the unified L1 as shared memory: two blocks of ~104 KB per SM
    cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kCholThreads, smem);
    return std::max(1, sms * std::min(std::max(per, 1), 4));
  }();
  return cached;
}

template <typename R>
cudaError_t launch_chol_batch(R* A, int lda, int nT, R* Linv, int* sync, uint32_t* status, LMState* lm,
                              int max_ctas, const Batch& bt, const uint32_t* order, cudaStream_t st) {
  const int n_tasks = chol_ntasks(nT);
  if (bt.G < 1 || (long long)n_tasks * bt.G > (1LL << 30)) return cudaErrorInvalidValue;
  if (order != nullptr && (bt.G > 4096 || n_tasks > (1 << 20))) return cudaErrorInvalidValue;
  const size_t smem = sizeof(R) * (6 * kNB) * Pitch<R>::value;  // two (X, Y, output) buffer triples
  int grid = std::min<long long>(chol_batch_grid<R>(smem), (long long)n_tasks * bt.G);
  if (max_ctas > 0) grid = std::min(grid, max_ctas);
  // every job's counters: rows of the reset length at the job stride
  const size_t row = sizeof(int) * chol_factor_reset_ints(nT);
  cudaError_t e = bt.G == 1 ? cudaMemsetAsync(sync, 0, row, st) : cudaMemset2DAsync(sync, bt.js, 0, row, bt.G, st);
  if (e != cudaSuccess) return e;
  k_chol_batch<R><<<grid, kCholThreads, smem, st>>>(A, lda, nT, Linv, n_tasks, bt.G, bt.js, order, sync, status,
                                                     lm);
  return cudaGetLastError();
}
template cudaError_t launch_chol_batch<float>(float*, int, int, float*, int*, uint32_t*, LMState*, int,
                                              const Batch&, const uint32_t*, cudaStream_t);
template cudaError_t launch_chol_batch<double>(double*, int, int, double*, int*, uint32_t*, LMState*, int,
                                               const Batch&, const uint32_t*, cudaStream_t);

// The combined task list of a batch's factorisations, the jobs staggered
// over a window of W jobs.  Job g's task t (of n per job) gets the key
// (t + 1) W + g n, i.e. its progress through its own list plus g / W of a
// list, and the combined list is sorted by (key, job): job g starts when
// job g - W is about to finish, so about W jobs are in flight at once, in
// different phases (one job's chain-bound last panels beside another's
// work-rich first ones), and only their matrices are being read.  Within a
// job the key grows with t, so every job keeps its own order.  The position
// of (g, t) counts, for every job g', the tasks with a smaller key (ties:
// the lower job first), in O(G).
__host__ __device__ int batch_order_pos(int n, int G, int W, int g, int t) {
  long long pos = 0;
  for (int h = 0; h < G; ++h) {
    // tasks t' of job h with (t' + 1) W < D, and one with (t' + 1) W == D
    const long long D = (long long)(t + 1) * W + (long long)(g - h) * n;
    if (D > W) pos += std::min<long long>(n, (D - 1) / W);
    if (h < g && D % W == 0 && D / W >= 1 && D / W <= n) pos += 1;
  }
  return (int)pos;
}

__global__ void k_batch_order(int n, int G, int W, uint32_t* __restrict__ order) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)n * G) return;
  const int g = (int)(i / n), t = (int)(i % n);
  const int p = batch_order_pos(n, G, W, g, t);
  if (p >= 0 && (long long)p < (long long)n * G) order[p] = ((uint32_t)g << 20) | (uint32_t)t;
}

bool batch_order_ok(int nT, int G) { return G >= 1 && G <= 4096 && chol_ntasks(nT) <= (1 << 20); }

cudaError_t launch_batch_order(int nT, int G, int W, uint32_t* order, cudaStream_t st) {
  if (!batch_order_ok(nT, G) || W < 1 || W > (1 << 20)) return cudaErrorInvalidValue;
  const long long total = (long long)chol_ntasks(nT) * G;
  k_batch_order<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(chol_ntasks(nT), G, W, order);
  return cudaGetLastError();
}

// ---- triangular solves ------------------------------------------------------------------------

// Asynchronous copy of one 64x64 tile into shared memory as one commit group.
template <typename R>
__device__ __forceinline__ void tile_async(R* sm, const R* g, int lda) {
  copy_tile_async(sm, g, lda);
  async_commit();
}
__device__ __forceinline__ void async_commit_empty() { async_commit(); }

// Tile-vector products on a 64x64 tile in shared memory (pitch 64 + 16
// bytes), laid out so that each quarter-warp's 16-byte loads hit all 32
// banks once.
//
// mv_rows: out[r] = sum_m T[r][m] v[m].  The quad of lanes 4r..4r+3 owns
// row r; lane `part` reads the row's 16-byte chunks part + 4u, rotated by
// three chunks on odd rows (odd rows start 4 banks further on, so the two
// rows of a quarter-warp then cover distinct banks).  Two shuffles combine
// the quad; every lane of it returns the row total.
__device__ __forceinline__ float mv_rows(const float* Tm, const float* v) {
  constexpr int LD = Pitch<float>::value;
  const int r = threadIdx.x >> 2, part = threadIdx.x & 3, rot = 3 * (r & 1);
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int ch = (part + 4 * u + rot) & 15;
    const float4 t = *reinterpret_cast<const float4*>(Tm + r * LD + 4 * ch);
    const float4 w = *reinterpret_cast<const float4*>(v + 4 * ch);
    s = fmaf(t.x, w.x, fmaf(t.y, w.y, fmaf(t.z, w.z, fmaf(t.w, w.w, s))));
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}
__device__ __forceinline__ double mv_rows(const double* Tm, const double* v) {
  constexpr int LD = Pitch<double>::value;
  const int r = threadIdx.x >> 2, part = threadIdx.x & 3, rot = 3 * (r & 1);
  double s = 0.0;
#pragma unroll
  for (int u = 0; u < 8; ++u) {  // 32 chunks of two doubles per row
    const int ch = (part + 4 * u + rot) & 31;
    const double2 t = *reinterpret_cast<const double2*>(Tm + r * LD + 2 * ch);
    const double2 w = *reinterpret_cast<const double2*>(v + 2 * ch);
    s = fma(t.x, w.x, fma(t.y, w.y, s));
  }
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  return s;
}

// mv_cols: out[c] = sum_m T[m][c] v[m] for the columns c = 4g..4g+3 of lane
// group g = tid / 16.  Lane mr of the group takes rows m = mr + 16k: a
// quarter-warp reads eight consecutive rows (4 banks apart) at one column
// offset.  Four butterfly rounds combine the group; every lane of it
// returns the four totals.
template <typename R>
__device__ __forceinline__ void mv_cols(const R* Tm, const R* v, R (&o)[4]) {
  constexpr int LD = Pitch<R>::value;
  const int g = threadIdx.x >> 4, mr = threadIdx.x & 15;
  R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int m = mr + 16 * k;
    const R* t = Tm + m * LD + 4 * g;
    const R w = v[m];
    if constexpr (sizeof(R) == 4) {
      const float4 q = *reinterpret_cast<const float4*>(t);
      a0 = fma((R)q.x, w, a0), a1 = fma((R)q.y, w, a1), a2 = fma((R)q.z, w, a2), a3 = fma((R)q.w, w, a3);
    } else {
      const double2 q0 = *reinterpret_cast<const double2*>(t);
      const double2 q1 = *reinterpret_cast<const double2*>(t + 2);
      a0 = fma((R)q0.x, w, a0), a1 = fma((R)q0.y, w, a1), a2 = fma((R)q1.x, w, a2), a3 = fma((R)q1.y, w, a3);
    }
  }
#pragma unroll
  for (int d = 1; d < 16; d <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, d);
    a1 += __shfl_xor_sync(0xffffffffu, a1, d);
    a2 += __shfl_xor_sync(0xffffffffu, a2, d);
    a3 += __shfl_xor_sync(0xffffffffu, a3, d);
  }
  o[0] = a0, o[1] = a1, o[2] = a2, o[3] = a3;
}

// C = A B for 64x64 tiles in shared memory (all with the tile pitch), 256
// threads with 4x4 outputs each: A is read as a broadcast per half-warp, B
// along contiguous rows.
template <typename R>
__device__ __forceinline__ void gemm_nn(R* C, const R* A, const R* B) {
  constexpr int LD = Pitch<R>::value;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  R acc[4][4] = {};
#pragma unroll 4
  for (int m = 0; m < kNB; ++m) {
    R a[4], b[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) a[u] = A[(ty + 16 * u) * LD + m];
#pragma unroll
    for (int u = 0; u < 4; ++u) b[u] = B[m * LD + tx + 16 * u];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int w = 0; w < 4; ++w) acc[u][w] = fma(a[u], b[w], acc[u][w]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int w = 0; w < 4; ++w) C[(ty + 16 * u) * LD + tx + 16 * w] = acc[u][w];
}

// Solved blocks of the substitution travel through global memory as tagged
// 64-bit words: (tag << 32) | 32 bits of the value, one word per float, two
// (high and low half) per double.  A word is written and read in one piece,
// so a reader that sees the tag of its launch and phase holds the value
// itself: no separate flag, no fence, one L2 round trip.  Tags are nonzero
// and unique per launch and phase, and the buffer is zeroed when a solve
// sequence starts, so neither stale words nor untouched memory can match.
__device__ __forceinline__ void put_tagged(uint64_t* w, float v, uint32_t tag) {
  __stcg(reinterpret_cast<unsigned long long*>(w), ((unsigned long long)tag << 32) | __float_as_uint(v));
}
__device__ __forceinline__ void put_tagged(uint64_t* w, double v, uint32_t tag) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  __stcg(reinterpret_cast<unsigned long long*>(w), ((unsigned long long)tag << 32) | (b >> 32));
  __stcg(reinterpret_cast<unsigned long long*>(w) + 1, ((unsigned long long)tag << 32) | (b & 0xffffffffull));
}
__device__ __forceinline__ unsigned long long ld_word(const uint64_t* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
// Waits (bounded) for the word(s) of one value carrying `tag`.
template <typename R>
__device__ bool get_tagged(const uint64_t* w, uint32_t tag, R& v, uint32_t* status) {
  constexpr int NW = sizeof(R) / 4;
  for (long it = 0; it < kSpinLimit; ++it) {
    const unsigned long long w0 = ld_word(w);
    const unsigned long long w1 = NW == 2 ? ld_word(w + 1) : w0;
    if ((uint32_t)(w0 >> 32) == tag && (uint32_t)(w1 >> 32) == tag) {
      if constexpr (NW == 1) v = (R)__uint_as_float((uint32_t)w0);
      else v = (R)__longlong_as_double((long long)((w0 << 32) | (w1 & 0xffffffffull)));
      return true;
    }
    if ((it & 63) == 63 && (ld_status(status) & SC_STATUS_TIMEOUT)) return false;
    if (it >= 32) __nanosleep(64);
  }
  atomicOr(status, SC_STATUS_TIMEOUT);
  return false;
}

// Block substitution, one task per tile row: FWD(i) y_i = Linv_ii (b_i -
// sum_{j<i} L_ij y_j), BWD(i) x_i = Linv_ii^T (y_i - sum_{j>i} L_ji^T x_j).
// Only the block that arrives last (y_{i-1}, resp. x_{i+1}) lies on the
// critical path, so a task folds everything else in before it comes:
//   FWD: M = Linv_ii L_{i,i-1},  z = Linv_ii (b_i - sum_{j<i-1} L_ij y_j),
//        then y_i = z - M y_{i-1}
//   BWD: N = L_{i+1,i} Linv_ii,  z = Linv_ii^T (y_i - sum_{j>i+1} L_ji^T x_j),
//        then x_i = z - N^T x_{i+1}
// which leaves one tile-vector product between a block's arrival and the
// publication of the next.  The other tiles stream through two shared
// buffers while the task waits for their blocks.  y_i and then x_i occupy
// the tagged words of row i (BWD(i) runs after every FWD task has finished,
// so no reader of y_i remains when x_i replaces it).
//
// A lock-step batch of G jobs takes the tasks of one combined list: task t
// is task t / G of job t mod G (dependencies stay earlier in the list); the
// counter is job 0's, every other pointer is the task's job's.
template <typename R>
__global__ void __launch_bounds__(kCholThreads) k_chol_solve(const R* __restrict__ A0, int lda, int nT,
                                                            const R* __restrict__ Linv0,
                                                            int n_tasks, int* sync0,
                                                            const double* __restrict__ b0,
                                                            uint64_t* __restrict__ yw0, double* __restrict__ x0,
                                                            int accumulate, uint32_t tag_fwd,
                                                            uint32_t* status0, const LMState* lm0, int G,
                                                            size_t js) {
  constexpr int LD = Pitch<R>::value;
  constexpr int NW = sizeof(R) / 4;  // tagged words per value
  const uint32_t tag_bwd = tag_fwd + 1;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* Tinv = reinterpret_cast<R*>(smraw);  // Linv_ii
  R* Tm = Tinv + kNB * LD;                // M (FWD) or N (BWD)
  R* B0 = Tm + kNB * LD;                  // the critical tile, then streamed tiles
  R* B1 = B0 + kNB * LD;
  R* vin = B1 + kNB * LD;
  __shared__ int s_task, s_ok;
  int* const counter = SyncView(sync0, nT).sctr;
  // the current task's job
  const R* A = A0;
  const R* Linv = Linv0;
  const double* b = b0;
  uint64_t* yw = yw0;
  double* x = x0;
  uint32_t* status = status0;
  const int tid = threadIdx.x;
  // forward: quad r = tid / 4 owns entry r (acc[0]); backward: lane group
  // g = tid / 16 owns entries 4g..4g+3
  auto acc_to_vin = [&](const R (&v)[4], bool fwd) {
    if (fwd) {
      if ((tid & 3) == 0) vin[tid >> 2] = v[0];
    } else if ((tid & 15) < 4) {
      const int e = tid & 15;
      vin[4 * (tid >> 4) + e] = e == 0 ? v[0] : e == 1 ? v[1] : e == 2 ? v[2] : v[3];
    }
  };
  auto fetch_block = [&](int row, uint32_t tag) {  // threads < 64: vin <- block `row`
    if (tid < kNB) {
      R v = 0;
      if (!get_tagged(yw + (size_t)NW * (row * kNB + tid), tag, v, status)) s_ok = 0;
      vin[tid] = v;
    }
  };
  for (;;) {
    __syncthreads();
    if (tid == 0) {
      s_task = atomicAdd(counter, 1);
      s_ok = 1;  // before the barrier: later failure reports cannot be lost
    }
    __syncthreads();
    const int tg = s_task;
    if (tg >= n_tasks * G) break;
    const int job = tg % G, t = tg / G;
    const LMState* lm = job_ptr(lm0, js, job);
    if (lm != nullptr && (lm->done | lm->notpd)) continue;
    A = job_ptr(A0, js, job);
    Linv = job_ptr(Linv0, js, job);
    b = job_ptr(b0, js, job);
    yw = job_ptr(yw0, js, job);
    x = job_ptr(x0, js, job);
    status = job_ptr(status0, js, job);
    const int4 tk = solve_task(nT, t);
    const int i = tk.y;
    const bool fwd = tk.x == T_FWD;
    const uint32_t tag_in = fwd ? tag_fwd : tag_bwd;  // tag of the blocks of other rows
    const bool crit = fwd ? i > 0 : i < nT - 1;       // a last-arriving block exists
    const int jc = fwd ? i - 1 : i + 1;               // ... and its row
    const int cnt = crit ? (fwd ? i - 1 : nT - 2 - i) : 0;  // the other off-diagonal tiles
    auto other_row = [&](int n) { return fwd ? n : nT - 1 - n; };
    auto other_tile = [&](int n) -> const R* {
      const int jj = other_row(n);
      return fwd ? A + (size_t)i * kNB * lda + (size_t)jj * kNB : A + (size_t)jj * kNB * lda + (size_t)i * kNB;
    };
    // group 0: Linv_ii and the critical tile; group 1: the first other tile
    copy_tile_async(Tinv, Linv + (size_t)i * kNB * kNB, kNB);
    if (crit)
      copy_tile_async(B0, fwd ? A + (size_t)i * kNB * lda + (size_t)jc * kNB : A + (size_t)jc * kNB * lda + (size_t)i * kNB,
                      lda);
    async_commit();
    if (cnt > 0) tile_async(B1, other_tile(0), lda);
    else async_commit_empty();
    R acc[4] = {0, 0, 0, 0};
    if (fwd) {
      acc[0] = (R)b[i * kNB + (tid >> 2)];
    } else {
      fetch_block(i, tag_fwd);  // y_i
      __syncthreads();
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[e] = vin[4 * (tid >> 4) + e];
    }
    async_wait_prev();  // group 0 has landed
    __syncthreads();
    if (crit) {
      if (fwd) gemm_nn(Tm, Tinv, B0);  // M = Linv_ii L_{i,i-1}
      else gemm_nn(Tm, B0, Tinv);      // N = L_{i+1,i} Linv_ii
    }
    for (int n = 0; n < cnt; ++n) {
      R* cur = (n & 1) ? B0 : B1;
      __syncthreads();  // every thread is done with vin and with the buffer refilled next
      if (n + 1 < cnt) tile_async((n & 1) ? B1 : B0, other_tile(n + 1), lda);
      else async_commit_empty();
      fetch_block(other_row(n), tag_in);
      async_wait_prev();
      __syncthreads();
      if (!s_ok) break;
      if (fwd) {
        acc[0] -= mv_rows(cur, vin);
      } else {
        R v[4];
        mv_cols(cur, vin, v);
#pragma unroll
        for (int e = 0; e < 4; ++e) acc[e] -= v[e];
      }
    }
    async_wait_all();
    if (!s_ok) break;
    // z = Linv_ii acc (FWD) or Linv_ii^T acc (BWD)
    __syncthreads();
    acc_to_vin(acc, fwd);
    __syncthreads();
    R o[4] = {0, 0, 0, 0};
    if (fwd) o[0] = mv_rows(Tinv, vin);
    else mv_cols(Tinv, vin, o);
    if (crit) {  // the critical block: one product
      __syncthreads();
      fetch_block(jc, tag_in);
      __syncthreads();
      if (!s_ok) break;
      if (fwd) {
        o[0] -= mv_rows(Tm, vin);
      } else {
        R v[4];
        mv_cols(Tm, vin, v);
#pragma unroll
        for (int e = 0; e < 4; ++e) o[e] -= v[e];
      }
    }
    if (fwd) {
      if ((tid & 3) == 0) put_tagged(yw + (size_t)NW * (i * kNB + (tid >> 2)), o[0], tag_fwd);
    } else if ((tid & 15) < 4) {
      const int e = tid & 15, r = 4 * (tid >> 4) + e;
      const R v = e == 0 ? o[0] : e == 1 ? o[1] : e == 2 ? o[2] : o[3];
      put_tagged(yw + (size_t)NW * (i * kNB + r), v, tag_bwd);
      x[i * kNB + r] = accumulate ? x[i * kNB + r] + (double)v : (double)v;
    }
  }
  async_wait_all();
}

static std::atomic<uint32_t> g_solve_launches{0};

template <typename R>
cudaError_t launch_chol_solve(const R* A, int lda, int nT, const R* Linv, int* sync,
                              const double* b, uint64_t* bwork, double* x, int accumulate,
                              uint32_t* status, const LMState* lm, cudaStream_t st, const Batch& bt) {
  int n_tasks = 2 * nT;
  if ((long long)n_tasks * bt.G > (1LL << 30)) return cudaErrorInvalidValue;
  size_t smem = sizeof(R) * (4 * kNB * Pitch<R>::value + kNB);
  static const bool attr_set = [&] {
    cudaFuncSetAttribute(reinterpret_cast<const void*>(&k_chol_solve<R>),
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return true;
  }();
  (void)attr_set;
  // tags 2e (forward) and 2e + 1 (backward), e >= 1, unique per launch
  const uint32_t e = (g_solve_launches.fetch_add(1, std::memory_order_relaxed) % 0x7ffffffeu) + 1;
  SyncView sv(sync, nT);
  cudaError_t err = cudaMemsetAsync(sv.sctr, 0, sizeof(int), st);
  if (err != cudaSuccess) return err;
  k_chol_solve<R><<<n_tasks * bt.G, kCholThreads, smem, st>>>(A, lda, nT, Linv, n_tasks, sync, b, bwork, x,
                                                              accumulate, 2 * e, status, lm, bt.G, bt.js);
  return cudaGetLastError();
}
template cudaError_t launch_chol_solve<float>(const float*, int, int, const float*, int*,
                                              const double*, uint64_t*, double*, int, uint32_t*,
                                              const LMState*, cudaStream_t, const Batch&);
template cudaError_t launch_chol_solve<double>(const double*, int, int, const double*, int*,
                                               const double*, uint64_t*, double*, int, uint32_t*,
                                               const LMState*, cudaStream_t, const Batch&);

}  // namespace sc
