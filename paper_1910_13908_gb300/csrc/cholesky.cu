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
// not stored)
// and wait, with a bounded spin, for the counters of the tiles they read.
// Every dependency of a task lies earlier in the list, so the earliest
// unfinished task can always run and the graph cannot deadlock; the list
// puts the next panel's POTRF/TRSM right after the updates they need
// (look-ahead of one panel), so the factorisation's critical path overlaps
// the bulk of the trailing updates.
//
// Tiles written by one SM and read by another are moved through L2 only
// (ld.global.cg / st.global.cg), and published with a fence followed by a
// release store of the tile's counter.
#include <algorithm>

#include "sc_common.cuh"

namespace sc {

enum TaskType { T_POTRF = 0, T_TRSM = 1, T_UPD = 2, T_FWD = 3, T_BWD = 4 };

// sync area (ints): [0] factor task counter, [1] solve task counter,
// upd[nT*nT], potrf_done[nT], trsm_done[nT*nT], fwd_done[nT], bwd_done[nT]
struct SyncView {
  int* fctr;
  int* sctr;
  int* upd;
  int* pdone;
  int* tdone;
  int* fdone;
  int* bdone;
  __host__ __device__ SyncView(int* s, int nT)
      : fctr(s), sctr(s + 1), upd(s + 2), pdone(s + 2 + nT * nT), tdone(s + 2 + nT * nT + nT),
        fdone(s + 2 + 2 * nT * nT + nT), bdone(s + 2 + 2 * nT * nT + 2 * nT) {}
};

int chol_sync_ints(int nT) { return 2 + 2 * nT * nT + 3 * nT; }
// ints from the start of the sync area that a factorisation resets
static int chol_factor_reset_ints(int nT) { return 2 + 2 * nT * nT + nT; }

// Task t of the factorisation list (decoded in O(nT), no list in memory):
//   POTRF(0), TRSM(1..nT-1, 0), then for each panel j = 0..nT-2:
//   UPDATE(j+1..nT-1, j+1, j)   -- the next panel column first
//   POTRF(j+1), TRSM(j+2..nT-1, j+1)
//   UPDATE(i, k, j) for k = j+2..nT-1, i = k..nT-1
// Returned as (type, i, k, j); type -1 past the end.
__host__ __device__ int4 chol_task(int nT, int t) {
  if (t == 0) return make_int4(T_POTRF, 0, 0, 0);
  t -= 1;
  if (t < nT - 1) return make_int4(T_TRSM, t + 1, 0, 0);
  t -= nT - 1;
  for (int j = 0; j + 1 < nT; ++j) {
    int m = nT - j - 1, m2 = nT - j - 2;
    int block = m + 1 + m2 + m2 * (m2 + 1) / 2;
    if (t >= block) {
      t -= block;
      continue;
    }
    if (t < m) return make_int4(T_UPD, j + 1 + t, j + 1, j);
    t -= m;
    if (t == 0) return make_int4(T_POTRF, j + 1, j + 1, j + 1);
    t -= 1;
    if (t < m2) return make_int4(T_TRSM, j + 2 + t, j + 1, j + 1);
    t -= m2;
    for (int k = j + 2; k < nT; ++k) {
      int c = nT - k;
      if (t < c) return make_int4(T_UPD, k + t, k, j);
      t -= c;
    }
  }
  return make_int4(-1, 0, 0, 0);
}

int chol_ntasks(int nT) {
  int n = nT;  // POTRF(0) + TRSM(1..nT-1, 0)
  for (int j = 0; j + 1 < nT; ++j) {
    int m = nT - j - 1, m2 = nT - j - 2;
    n += m + 1 + m2 + m2 * (m2 + 1) / 2;
  }
  return n;
}

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
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint32_t ld_status(const uint32_t* p) {
  return *reinterpret_cast<const volatile uint32_t*>(p);
}

// Waits until *p >= v.  Gives up (returns false) after kSpinLimit polls or as
// soon as another CTA has recorded a timeout.
__device__ bool wait_ge(const int* p, int v, uint32_t* status) {
  for (long it = 0; it < kSpinLimit; ++it) {
    if (ld_acquire(p) >= v) return true;
    if ((it & 63) == 63 && (ld_status(status) & SC_STATUS_TIMEOUT)) return false;
    __nanosleep(it < 16 ? 32 : 200);
  }
  atomicOr(status, SC_STATUS_TIMEOUT);
  return false;
}

// ---- tile helpers --------------------------------------------------------------------------

constexpr int LD = kNB + 1;  // padded shared-memory row

template <typename R>
__device__ __forceinline__ void load_tile(R* sm, const R* g, int lda) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    sm[r * LD + c] = __ldcg(g + (size_t)r * lda + c);
  }
}
template <typename R>
__device__ __forceinline__ void store_tile(R* g, int lda, const R* sm) {
  for (int e = threadIdx.x; e < kNB * kNB; e += blockDim.x) {
    int r = e >> 6, c = e & 63;
    __stcg(g + (size_t)r * lda + c, sm[r * LD + c]);
  }
}

// acc[a][b] = sum_m X[ty+16a][m] Y[tx+16b][m]   (X Y^T on 64x64 tiles)
template <typename R>
__device__ __forceinline__ void gemm_nt(R acc[4][4], const R* X, const R* Y) {
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0;
#pragma unroll 4
  for (int m = 0; m < kNB; ++m) {
    R x[4], y[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) x[a] = X[(ty + 16 * a) * LD + m];
#pragma unroll
    for (int b = 0; b < 4; ++b) y[b] = Y[(tx + 16 * b) * LD + m];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = fma(x[a], y[b], acc[a][b]);
  }
}

// In-place Cholesky of the 64x64 tile in sm (lower part read), writing L
// (upper part zeroed); then Linv = L^-1 into sv.  Non-positive pivots are
// replaced by 1 and reported through *bad.
template <typename R>
__device__ void potrf_tile(R* sm, R* sv, R* piv, int* bad) {
  int tid = threadIdx.x;
  int r = tid >> 2, cb = tid & 3;
  for (int c = 0; c < kNB; ++c) {
    R p = sm[c * LD + c];
    if (!(p > (R)0)) {
      p = (R)1;
      if (tid == 0) *bad = 1;
    }
    if (tid == 0) piv[c] = p;
    if (r > c) {
      R arc = sm[r * LD + c] / p;
#pragma unroll
      for (int u = 0; u < 16; ++u) {
        int cc = cb + 4 * u;
        if (cc > c && cc <= r) sm[r * LD + cc] -= arc * sm[cc * LD + c];
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    int cc = cb + 4 * u;
    R v;
    if (cc < r) v = sm[r * LD + cc] / sqrt(piv[cc]);
    else if (cc == r) v = sqrt(piv[r]);
    else v = 0;
    sm[r * LD + cc] = v;
  }
  __syncthreads();
  // Linv: column c = tid/4 by forward substitution, 4 lanes per column
  int c = tid >> 2, part = tid & 3;
  for (int rr = 0; rr < kNB; ++rr) {
    R s = 0;
    if (rr > c)
      for (int m = c + part; m < rr; m += 4) s += sm[rr * LD + m] * sv[m * LD + c];
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    s += __shfl_xor_sync(0xffffffffu, s, 2);
    if (part == 0) {
      R v = 0;
      if (rr == c) v = (R)1 / sm[rr * LD + rr];
      else if (rr > c) v = -s / sm[rr * LD + rr];
      sv[rr * LD + c] = v;
    }
    __syncwarp();
  }
  __syncthreads();
}

// ---- factorisation ---------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(kCholThreads) k_chol(R* __restrict__ A, int lda, int nT,
                                                      R* __restrict__ Linv, int n_tasks,
                                                      int* sync, uint32_t* status, LMState* lm) {
  if (lm != nullptr && lm->done) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* s0 = reinterpret_cast<R*>(smraw);
  R* s1 = s0 + kNB * LD;
  R* piv = s1 + kNB * LD;
  __shared__ int s_task, s_ok, s_bad;
  SyncView sv(sync, nT);
  for (;;) {
    if (threadIdx.x == 0) {
      s_task = atomicAdd(sv.fctr, 1);
      s_bad = 0;
    }
    __syncthreads();
    int t = s_task;
    if (t >= n_tasks) break;
    int4 tk = chol_task(nT, t);
    int i = tk.y, k = tk.z, j = tk.w;
    if (threadIdx.x == 0) {
      bool ok = true;
      if (tk.x == T_POTRF) {
        ok = wait_ge(sv.upd + j * nT + j, j, status);
      } else if (tk.x == T_TRSM) {
        ok = wait_ge(sv.pdone + j, 1, status) && wait_ge(sv.upd + i * nT + j, j, status);
      } else {
        ok = wait_ge(sv.tdone + i * nT + j, 1, status) && wait_ge(sv.tdone + k * nT + j, 1, status) &&
             wait_ge(sv.upd + i * nT + k, j, status);
      }
      s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) {
      if (threadIdx.x == 0 && lm != nullptr) lm->notpd = 1;
      break;
    }
    if (tk.x == T_POTRF) {
      R* Ajj = A + (size_t)j * kNB * lda + (size_t)j * kNB;
      load_tile(s0, Ajj, lda);
      __syncthreads();
      potrf_tile(s0, s1, piv, &s_bad);
      store_tile(Ajj, lda, s0);
      store_tile(Linv + (size_t)j * kNB * kNB, kNB, s1);  // Linv tiles: leading dim 64
      __syncthreads();
      if (threadIdx.x == 0) {
        if (s_bad) {
          atomicOr(status, SC_STATUS_NOTPD);
          if (lm != nullptr) lm->notpd = 1;
        }
        __threadfence();
        st_release(sv.pdone + j, 1);
      }
    } else if (tk.x == T_TRSM) {
      R* Aij = A + (size_t)i * kNB * lda + (size_t)j * kNB;
      load_tile(s0, Aij, lda);
      load_tile(s1, Linv + (size_t)j * kNB * kNB, kNB);
      __syncthreads();
      R acc[4][4];
      gemm_nt(acc, s0, s1);
      int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) __stcg(Aij + (size_t)(ty + 16 * a) * lda + tx + 16 * b, acc[a][b]);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(sv.tdone + i * nT + j, 1);
      }
    } else {
      const R* Lij = A + (size_t)i * kNB * lda + (size_t)j * kNB;
      const R* Lkj = A + (size_t)k * kNB * lda + (size_t)j * kNB;
      R* Aik = A + (size_t)i * kNB * lda + (size_t)k * kNB;
      load_tile(s0, Lij, lda);
      load_tile(s1, Lkj, lda);
      __syncthreads();
      R acc[4][4];
      gemm_nt(acc, s0, s1);
      int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          R* p = Aik + (size_t)(ty + 16 * a) * lda + tx + 16 * b;
          __stcg(p, __ldcg(p) - acc[a][b]);
        }
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        st_release(sv.upd + i * nT + k, j + 1);
      }
    }
  }
}

template <typename R>
static int chol_grid(const void* fn, size_t smem) {
  static int cached[2] = {0, 0};
  int slot = sizeof(R) == 8 ? 1 : 0;
  if (cached[slot] == 0) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kCholThreads, smem);
    cached[slot] = std::max(1, sms * std::min(std::max(per, 1), 4));
  }
  return cached[slot];
}

template <typename R>
cudaError_t launch_chol(R* A, int lda, int nT, R* Linv, int* sync, uint32_t* status, LMState* lm,
                        cudaStream_t st) {
  int n_tasks = chol_ntasks(nT);
  size_t smem = sizeof(R) * (2 * kNB * LD + kNB);
  const void* fn = reinterpret_cast<const void*>(&k_chol<R>);
  int grid = std::min(chol_grid<R>(fn, smem), n_tasks);
  cudaError_t e = cudaMemsetAsync(sync, 0, sizeof(int) * chol_factor_reset_ints(nT), st);
  if (e != cudaSuccess) return e;
  k_chol<R><<<grid, kCholThreads, smem, st>>>(A, lda, nT, Linv, n_tasks, sync, status, lm);
  return cudaGetLastError();
}
template cudaError_t launch_chol<float>(float*, int, int, float*, int*, uint32_t*, LMState*,
                                        cudaStream_t);
template cudaError_t launch_chol<double>(double*, int, int, double*, int*, uint32_t*, LMState*,
                                         cudaStream_t);

// ---- triangular solves ------------------------------------------------------------------------

// out[r] = sum_m T[r][m] v[m] (trans = 0) or sum_m T[m][r] v[m] (trans = 1) for a
// 64x64 tile in shared memory; 4 threads per r, combined through red[4][64].
template <typename R>
__device__ __forceinline__ R tile_matvec(const R* Tm, const R* v, R* red, int trans) {
  int r = threadIdx.x & 63, part = threadIdx.x >> 6;
  R s = 0;
#pragma unroll 4
  for (int m = 16 * part; m < 16 * part + 16; ++m)
    s += (trans ? Tm[m * LD + r] : Tm[r * LD + m]) * v[m];
  red[part * kNB + r] = s;
  __syncthreads();
  R tot = red[r] + red[kNB + r] + red[2 * kNB + r] + red[3 * kNB + r];
  __syncthreads();
  return tot;
}

template <typename R>
__global__ void __launch_bounds__(kCholThreads) k_chol_solve(const R* __restrict__ A, int lda, int nT,
                                                            const R* __restrict__ Linv,
                                                            int n_tasks, int* sync,
                                                            const double* __restrict__ b,
                                                            R* __restrict__ yw, double* __restrict__ x,
                                                            int accumulate, uint32_t* status,
                                                            const LMState* lm) {
  if (lm != nullptr && (lm->done | lm->notpd)) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  R* tile = reinterpret_cast<R*>(smraw);
  R* vin = tile + kNB * LD;
  R* red = vin + kNB;
  __shared__ int s_task, s_ok;
  SyncView sv(sync, nT);
  int r = threadIdx.x & 63, part = threadIdx.x >> 6;
  for (;;) {
    if (threadIdx.x == 0) s_task = atomicAdd(sv.sctr, 1);
    __syncthreads();
    int t = s_task;
    if (t >= n_tasks) break;
    int4 tk = solve_task(nT, t);
    int i = tk.y;
    R acc = 0;
    bool fwd = tk.x == T_FWD;
    if (fwd) {
      acc = (R)b[i * kNB + r];
    } else {
      if (threadIdx.x == 0) s_ok = wait_ge(sv.fdone + i, 1, status);
      __syncthreads();
      if (!s_ok) break;
      acc = __ldcg(yw + i * kNB + r);
    }
    int j0 = fwd ? 0 : nT - 1, j1 = fwd ? i : i, dj = fwd ? 1 : -1;
    bool ok = true;
    for (int jj = j0; jj != j1; jj += dj) {
      if (threadIdx.x == 0) s_ok = wait_ge((fwd ? sv.fdone : sv.bdone) + jj, 1, status);
      __syncthreads();
      if (!s_ok) {
        ok = false;
        break;
      }
      if (fwd) load_tile(tile, A + (size_t)i * kNB * lda + (size_t)jj * kNB, lda);
      else load_tile(tile, A + (size_t)jj * kNB * lda + (size_t)i * kNB, lda);
      if (threadIdx.x < kNB) vin[threadIdx.x] = __ldcg(yw + jj * kNB + threadIdx.x);
      __syncthreads();
      acc -= tile_matvec(tile, vin, red, fwd ? 0 : 1);
    }
    if (!ok) break;
    load_tile(tile, Linv + (size_t)i * kNB * kNB, kNB);
    if (part == 0) vin[r] = acc;
    __syncthreads();
    R out = tile_matvec(tile, vin, red, fwd ? 0 : 1);
    if (part == 0) {
      __stcg(yw + i * kNB + r, out);
      if (!fwd) {
        double o = (double)out;
        x[i * kNB + r] = accumulate ? x[i * kNB + r] + o : o;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      st_release((fwd ? sv.fdone : sv.bdone) + i, 1);
    }
  }
}

template <typename R>
cudaError_t launch_chol_solve(const R* A, int lda, int nT, const R* Linv, int* sync,
                              const double* b, R* bwork, double* x, int accumulate,
                              uint32_t* status, const LMState* lm, cudaStream_t st) {
  int n_tasks = 2 * nT;
  size_t smem = sizeof(R) * (kNB * LD + kNB + 4 * kNB);
  SyncView sv(sync, nT);
  // reset the solve counter and the fwd/bwd flags
  cudaError_t e = cudaMemsetAsync(sv.sctr, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(sv.fdone, 0, sizeof(int) * 2 * nT, st);
  if (e != cudaSuccess) return e;
  int grid = std::min(n_tasks, 2 * nT);
  k_chol_solve<R><<<grid, kCholThreads, smem, st>>>(A, lda, nT, Linv, n_tasks, sync, b, bwork, x,
                                                    accumulate, status, lm);
  return cudaGetLastError();
}
template cudaError_t launch_chol_solve<float>(const float*, int, int, const float*, int*,
                                              const double*, float*, double*, int, uint32_t*,
                                              const LMState*, cudaStream_t);
template cudaError_t launch_chol_solve<double>(const double*, int, int, const double*, int*,
                                               const double*, double*, double*, int, uint32_t*,
                                               const LMState*, cudaStream_t);

}  // namespace sc
