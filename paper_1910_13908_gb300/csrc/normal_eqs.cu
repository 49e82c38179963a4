// Step (c): the Gauss-Newton matrix J^T J of one cluster, written densely
// (8N x 8N) for the Cholesky factorisation, and the float64 product
// (J^T J + mu I) x used by the iterative refinement of the float32 solve.
//
// With the unpolarised coherency c Id, a change dJ of the Jones changes the
// model of baseline so by c (dJ_s J_o^H + J_s dJ_o^H), and J^T applied to
// that change gives, for station s,
//     (J^T J dJ)_s = dJ_s H_s + J_s sum_{o != s} w_so dJ_o^H J_o,
//     H_s = sum_{o != s} w_so J_o^H J_o,   w_so = sum_{t,f} |c_so(t,f)|^2.
// Written in the real parameters theta[8s + 4i + 2j + x] (x = 0 real,
// 1 imaginary part of J_s[i][j]) the 8x8 blocks are
//   off-diagonal (s, o), Z = w_so J_s[i][a] J_o[b][j], row (x,i,j), col (y,b,a):
//       (0,0): Re Z   (1,0): Im Z   (0,1): Im Z   (1,1): -Re Z
//   diagonal s, Hd = H_s + mu I (LM damping), row (x,i,j), col (y,i',a), i' = i:
//       (0,0): Re Hd[a][j]   (1,0): Im Hd[a][j]   (0,1): -Im Hd[a][j]   (1,1): Re Hd[a][j]
// (the real form of dJ_s -> dJ_s Hd and dJ_o -> w J_s dJ_o^H J_o).  The
// matrix depends on the data only through w, so it is assembled in O(P^2)
// without touching the visibilities; its cost is the matrix write itself.
#include "sc_common.cuh"

namespace sc {

template <typename R>
__device__ __forceinline__ cx<R> jent(const R* __restrict__ J, int s, int i, int j) {
  const R* p = J + 8 * s + 4 * i + 2 * j;
  return {p[0], p[1]};
}

__device__ __forceinline__ void st4(float* d, const float* v) {
  *reinterpret_cast<float4*>(d) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void st4(double* d, const double* v) {
  reinterpret_cast<double2*>(d)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(d)[1] = make_double2(v[2], v[3]);
}

// J: the Jones in R (rounded once by the LM trial step in float32), so that
// the float64 pipe, slow on this GPU, converts nothing per element.
template <typename R>
__global__ void __launch_bounds__(256) k_assemble(int N, int lda, int Ppad, const R* __restrict__ w,
                                                  const R* __restrict__ J,
                                                  const double* __restrict__ H,
                                                  const LMState* __restrict__ lm, R* __restrict__ A,
                                                  int damp, int full, size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm != nullptr && lm->done) return;
  w = job_ptr(w, js, job);
  J = job_ptr(J, js, job);
  H = job_ptr(H, js, job);
  A = job_ptr(A, js, job);
  int P = 8 * N;
  int row = blockIdx.y;
  int col0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (col0 >= Ppad) return;
  if (!full && col0 > row) return;  // lower triangle (+ the 4-wide group on the diagonal)
  R out[4];
  if (row >= P) {
#pragma unroll
    for (int u = 0; u < 4; ++u) out[u] = (col0 + u == row) ? (R)1 : (R)0;
  } else {
    int s = row >> 3, rr = row & 7;
    int i = rr >> 2, j = (rr >> 1) & 1, x = rr & 1;
    int o = col0 >> 3;
    if (col0 >= P) {
#pragma unroll
      for (int u = 0; u < 4; ++u) out[u] = 0;
    } else if (o != s) {
      int64_t b = s < o ? bl_index(s, o, N) : bl_index(o, s, N);
      R wb = w[b];
      int bb = (col0 & 7) >> 2;  // row index b of J_o for these 4 columns
      cx<R> Job = jent<R>(J, o, bb, j);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int cc = (col0 + u) & 3;
        int a = cc >> 1, y = cc & 1;
        cx<R> Z = jent<R>(J, s, i, a) * Job;
        Z = scale(Z, wb);
        R v;
        if (x == 0 && y == 0) v = Z.re;
        else if (x == 1 && y == 0) v = Z.im;
        else if (x == 0 && y == 1) v = Z.im;
        else v = -Z.re;
        out[u] = v;
      }
    } else {
      const R mu = (damp && lm != nullptr) ? (R)lm->mu : (R)0;
      const double* h = H + 4 * s;
      int ip = (col0 & 7) >> 2;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        int cc = (col0 + u) & 3;
        int a = cc >> 1, y = cc & 1;
        R v = 0;
        if (ip == i) {
          cx<R> hd;
          if (a == 0 && j == 0) hd = {(R)h[0] + mu, (R)0};
          else if (a == 1 && j == 1) hd = {(R)h[1] + mu, (R)0};
          else if (a == 0 && j == 1) hd = {(R)h[2], (R)h[3]};
          else hd = {(R)h[2], -(R)h[3]};
          if (x == 0 && y == 0) v = hd.re;
          else if (x == 1 && y == 0) v = hd.im;
          else if (x == 0 && y == 1) v = -hd.im;
          else v = hd.re;
        }
        out[u] = v;
      }
    }
  }
  // lda and col0 are multiples of 4, so the 4 values are one aligned vector
  R* dst = A + (size_t)row * lda + col0;
  if (col0 < lda) st4(dst, out);
}

__global__ void k_round_jones(const double* __restrict__ J, float* __restrict__ Jf, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) Jf[k] = (float)J[k];
}

cudaError_t launch_round_jones(const double* J, float* Jf, int n, cudaStream_t st) {
  k_round_jones<<<(n + 255) / 256, 256, 0, st>>>(J, Jf, n);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_assemble(const Shape& s, int lda, int Ppad, const R* w, const R* J,
                            const double* H, const LMState* lm, R* A, bool damp, bool full,
                            cudaStream_t st, const Batch& bt) {
  int groups = (Ppad + 3) / 4;
  dim3 grd((groups + 127) / 128, Ppad, bt.G);
  k_assemble<R><<<grd, 128, 0, st>>>(s.N, lda, Ppad, w, J, H, lm, A, damp ? 1 : 0, full ? 1 : 0, bt.js);
  return cudaGetLastError();
}
template cudaError_t launch_assemble<float>(const Shape&, int, int, const float*, const float*,
                                            const double*, const LMState*, float*, bool, bool,
                                            cudaStream_t, const Batch&);
template cudaError_t launch_assemble<double>(const Shape&, int, int, const double*, const double*,
                                             const double*, const LMState*, double*, bool, bool,
                                             cudaStream_t, const Batch&);

// Ones on the diagonal of rows n..Ppad-1 of a zeroed padded matrix, so that
// the padding factorises as the identity.
template <typename R>
__global__ void k_pad_identity(R* __restrict__ A, int lda, int n, int Ppad) {
  const int r = n + blockIdx.x * blockDim.x + threadIdx.x;
  if (r < Ppad) A[(size_t)r * lda + r] = (R)1;
}

template <typename R>
cudaError_t launch_pad_identity(R* A, int Ppad, int n, cudaStream_t st) {
  if (n >= Ppad) return cudaSuccess;
  k_pad_identity<R><<<1, 64, 0, st>>>(A, Ppad, n, Ppad);
  return cudaGetLastError();
}
template cudaError_t launch_pad_identity<float>(float*, int, int, cudaStream_t);
template cudaError_t launch_pad_identity<double>(double*, int, int, cudaStream_t);

// ---- float64 refinement residual r = g - (J^T J + mu I) x ---------------------------------

__device__ __forceinline__ m22<double> ld_m22(const double* p) {
  return {{p[0], p[1]}, {p[2], p[3]}, {p[4], p[5]}, {p[6], p[7]}};
}

// r = g - (J^T J + mu I) x.  With X_s the 2x2 complex form of x's station
// block and Y_o = X_o^H J_o, the product's station block is
//     X_s (H_s + mu I) + J_s sum_{o != s} w_so Y_o,
// so Y is formed once per station (k_refine_prep) and each station then
// needs 8 multiply-adds per other station: one block of kRefineWarps warps
// per station, the warps' lanes striding over the other stations, a fixed
// butterfly within each warp and a fixed-order sum over the warps.
__global__ void __launch_bounds__(256) k_refine_prep(int N, const double* __restrict__ J,
                                                     const double* __restrict__ x,
                                                     const LMState* __restrict__ lm, double* __restrict__ Y,
                                                     size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm->done | lm->notpd) return;
  J = job_ptr(J, js, job);
  x = job_ptr(x, js, job);
  Y = job_ptr(Y, js, job);
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= N) return;
  const m22<double> t = h_mul(ld_m22(x + 8 * o), load_jones<double>(J, o));
  double* y = Y + 8 * o;
  y[0] = t.a.re, y[1] = t.a.im, y[2] = t.b.re, y[3] = t.b.im;
  y[4] = t.c.re, y[5] = t.c.im, y[6] = t.d.re, y[7] = t.d.im;
}

constexpr int kRefineWarps = 4;
template <typename R>
__global__ void __launch_bounds__(32 * kRefineWarps) k_refine_residual(int N, const R* __restrict__ w,
                                                         const double* __restrict__ J,
                                                         const double* __restrict__ H,
                                                         const double* __restrict__ g,
                                                         const double* __restrict__ x,
                                                         const double* __restrict__ Y,
                                                         const LMState* __restrict__ lm,
                                                         double* __restrict__ r, size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm->done | lm->notpd) return;
  w = job_ptr(w, js, job);
  J = job_ptr(J, js, job);
  H = job_ptr(H, js, job);
  g = job_ptr(g, js, job);
  x = job_ptr(x, js, job);
  Y = job_ptr(Y, js, job);
  r = job_ptr(r, js, job);
  __shared__ double part[kRefineWarps][8];
  const int s = blockIdx.x, lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  double k[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int o = threadIdx.x; o < N; o += 32 * kRefineWarps) {
    if (o == s) continue;
    const double wb = (double)w[s < o ? bl_index(s, o, N) : bl_index(o, s, N)];
    const double2* y = reinterpret_cast<const double2*>(Y + 8 * o);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double2 v = y[u];
      k[2 * u] = fma(wb, v.x, k[2 * u]);
      k[2 * u + 1] = fma(wb, v.y, k[2 * u + 1]);
    }
  }
#pragma unroll
  for (int u = 0; u < 8; ++u) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) k[u] += __shfl_xor_sync(0xffffffffu, k[u], d);
  }
  if (lane == 0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) part[wi][u] = k[u];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      double t = part[0][u];
      for (int v = 1; v < kRefineWarps; ++v) t += part[v][u];
      k[u] = t;
    }
    const m22<double> Ks = {{k[0], k[1]}, {k[2], k[3]}, {k[4], k[5]}, {k[6], k[7]}};
    const double* h = H + 4 * s;
    const double mu = lm->mu;
    const m22<double> Hd = {{h[0] + mu, 0.0}, {h[2], h[3]}, {h[2], -h[3]}, {h[1] + mu, 0.0}};
    const m22<double> y = mul(ld_m22(x + 8 * s), Hd) + mul(load_jones<double>(J, s), Ks);
    const double y8[8] = {y.a.re, y.a.im, y.b.re, y.b.im, y.c.re, y.c.im, y.d.re, y.d.im};
    for (int i = 0; i < 8; ++i) r[8 * s + i] = g[8 * s + i] - y8[i];
  }
}

template <typename R>
cudaError_t launch_refine_residual(const Shape& s, const R* w, const double* J, const double* H,
                                   const double* g, const double* x, const LMState* lm,
                                   double* Y, double* r, cudaStream_t st, const Batch& bt) {
  k_refine_prep<<<dim3((s.N + 255) / 256, 1, bt.G), 256, 0, st>>>(s.N, J, x, lm, Y, bt.js);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_refine_residual<R><<<dim3(s.N, 1, bt.G), 32 * kRefineWarps, 0, st>>>(s.N, w, J, H, g, x, Y, lm, r, bt.js);
  return cudaGetLastError();
}
template cudaError_t launch_refine_residual<float>(const Shape&, const float*, const double*,
                                                   const double*, const double*, const double*,
                                                   const LMState*, double*, double*, cudaStream_t, const Batch&);
template cudaError_t launch_refine_residual<double>(const Shape&, const double*, const double*,
                                                    const double*, const double*, const double*,
                                                    const LMState*, double*, double*, cudaStream_t, const Batch&);

}  // namespace sc
