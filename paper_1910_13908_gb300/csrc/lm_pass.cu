// Step (b): streaming passes over the visibilities of one cluster.  k_pass
// forms residuals and per-baseline sums: the residual call and its cost, and
// the running residual of SAGE.  The LM loop works from per-baseline
// statistics instead (lm_stats.cu).
//
// For baseline pq and coherency c = C_pq(t,f) the model is c J_p J_q^H.  The
// pass forms, per visibility,
//     X = Xin (+ c G_old)       (E-step data from the running residual)
//     r = X - c G,   G = J_p J_q^H
// and accumulates per baseline (over the timeslots of a chunk and all
// channels) cost_b = sum |r|_F^2 and rho_b = sum conj(c) r.  The gradient of
// the cost with respect to J_p is then -2 rho_b J_q and with respect to J_q
// -2 rho_b^H J_p, so J^T r of station s is sum_o rho J_o (s = p) or
// rho^H J_o (s = q).  The diagonal 8x8 block of J^T J of station s is the
// real form of dJ_s -> dJ_s H_s with H_s = sum_o w_so J_o^H J_o, and
// w_so = sum |c_so|^2 (see normal_eqs.cu).
//
// The running residual's update in float32 (no statistics) has its own
// kernel, k_pass_col32, below.
//
// Memory: one thread per (baseline, timeslot chunk); consecutive threads take
// consecutive baselines, whose [F][2][2] complex blocks are contiguous in the
// [T][B][F][2][2] layout, so every warp streams contiguous memory.
#include <algorithm>

#include "sc_common.cuh"

namespace sc {

template <typename R, int FL>
__global__ void __launch_bounds__(256) k_pass(int N, int T, int F, int64_t B, int nchunk, int tchunk,
                                              const R* Xin, const R* __restrict__ C,
                                              const double* __restrict__ J_old,
                                              const double* __restrict__ J_cur, R* Rout,
                                              R* __restrict__ stat_cost, R* __restrict__ stat_rho,
                                              const LMState* __restrict__ lm) {
  if (lm != nullptr && (lm->done | lm->skip)) return;
  const int64_t n_items = (int64_t)nchunk * B;
  // grid-stride over (chunk, baseline) items: the grid is sized to the
  // resident blocks, so no partly filled last wave
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_items;
       idx += (int64_t)gridDim.x * blockDim.x) {
  int chunk = (int)(idx / B);
  int64_t b = idx - (int64_t)chunk * B;
  int p, q;
  bl_pair(b, N, p, q);
  m22<R> G = mzero<R>(), Go = mzero<R>();
  if (FL & P_SUB) G = mul_h(load_jones<R>(J_cur, p), load_jones<R>(J_cur, q));
  if (FL & P_OLD) Go = mul_h(load_jones<R>(J_old, p), load_jones<R>(J_old, q));
  R cost = 0;
  m22<R> rho = mzero<R>();
  int t0 = chunk * tchunk, t1 = min(T, t0 + tchunk);
#pragma unroll 2
  for (int t = t0; t < t1; ++t) {
    size_t v0 = ((size_t)t * B + b) * F;
#pragma unroll 4
    for (int f = 0; f < F; ++f) {
      size_t v = v0 + f;
      m22<R> x;
      if (FL & P_WRITE_R) {
        // may run in place (Rout == Xin): plain loads
        const R* px = Xin + 8 * v;
        x = {{px[0], px[1]}, {px[2], px[3]}, {px[4], px[5]}, {px[6], px[7]}};
      } else {
        x = ld_vis(Xin + 8 * v);
      }
      cx<R> c = ld_c(C + 2 * v);
      if (FL & P_OLD) x = x + smul(c, Go);
      if (FL & P_SUB) x = x - smul(c, G);
      if (FL & P_WRITE_R) st_vis(Rout + 8 * v, x);
      if (FL & P_STATS) {
        cost += frob2(x);
        rho.a = rho.a + cmulc(c, x.a);
        rho.b = rho.b + cmulc(c, x.b);
        rho.c = rho.c + cmulc(c, x.c);
        rho.d = rho.d + cmulc(c, x.d);
      }
    }
  }
  if (FL & P_STATS) {
    size_t o = (size_t)chunk * B + b;
    stat_cost[o] = cost;
    st_vis(stat_rho + 8 * o, rho);
  }
  }
}

template <typename R, int FL>
static cudaError_t go_pass(const Shape& s, const R* Xin, const R* C, const double* J_old,
                           const double* J_cur, R* Rout, R* stat_cost, R* stat_rho, int nchunk,
                           int tchunk, const LMState* lm, cudaStream_t st) {
  // resident blocks of this instantiation, computed once (thread-safe static)
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pass<R, FL>, 256, 0);
    return std::max(1, sms * std::max(per, 1));
  }();
  const int64_t n = (int64_t)nchunk * s.B;
  const unsigned grid = (unsigned)std::min<int64_t>((n + 255) / 256, resident);
  k_pass<R, FL><<<grid, 256, 0, st>>>(s.N, s.T, s.F, s.B, nchunk, tchunk, Xin, C, J_old, J_cur, Rout,
                                      stat_cost, stat_rho, lm);
  return cudaGetLastError();
}

// ---- the running residual's update in float32 ---------------------------------------------
//
// Without statistics, the pass is X + c G_old - c G per visibility
// (G_old only with P_OLD), G = J_p J_q^H, with the arithmetic of k_pass
// (the same expressions, so a residual is the same bits with or without
// its cost, and the mixed path's LM trajectories, which amplify any change
// of rounding, stay where they were).  What changes is the access: one
// thread owns one (baseline, channel) column of the [T][B][F][2][2] layout
// and walks its timeslots, so consecutive threads read consecutive 32-byte
// visibilities, G_old and G stay in registers, and the loads of several
// timeslots are issued before their stores (k_pass, one thread per
// (baseline, timeslot chunk), has one visibility in flight: the compiler
// cannot move a load above a store that may alias it).

template <int FL>
__global__ void __launch_bounds__(256) k_pass_col32(int N, int T, int F, int64_t B, const float* Xin,
                                                    const float* __restrict__ C, const double* __restrict__ J_old,
                                                    const double* __restrict__ J_cur, float* Rout) {
  const int64_t cols = B * F;
  for (int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; col < cols;
       col += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = col / F;
    int p, q;
    bl_pair(b, N, p, q);
    const m22<float> G = mul_h(load_jones<float>(J_cur, p), load_jones<float>(J_cur, q));
    m22<float> Go = mzero<float>();
    if (FL & P_OLD) Go = mul_h(load_jones<float>(J_old, p), load_jones<float>(J_old, q));
    // may run in place (Rout == Xin): plain loads.  The compiler cannot
    // move a load above a store that may alias it, so the loads of kTs
    // timeslots are written before their stores: kTs visibilities in
    // flight per thread.
    const float4* x = reinterpret_cast<const float4*>(Xin) + 2 * col;
    float4* o = reinterpret_cast<float4*>(Rout) + 2 * col;
    const float2* cp = reinterpret_cast<const float2*>(C) + col;
    constexpr int kTs = 4;
    auto update = [&](float4& u, float4& v, float2 cc) {
      m22<float> xv = {{u.x, u.y}, {u.z, u.w}, {v.x, v.y}, {v.z, v.w}};
      const cx<float> c = {cc.x, cc.y};
      if (FL & P_OLD) xv = xv + smul(c, Go);
      xv = xv - smul(c, G);
      u = make_float4(xv.a.re, xv.a.im, xv.b.re, xv.b.im);
      v = make_float4(xv.c.re, xv.c.im, xv.d.re, xv.d.im);
    };
    int t = 0;
    for (; t + kTs <= T; t += kTs) {
      float4 u[kTs], v[kTs];
      float2 c[kTs];
#pragma unroll
      for (int k = 0; k < kTs; ++k) {
        const size_t tv = (size_t)(t + k) * cols;
        u[k] = x[2 * tv];
        v[k] = x[2 * tv + 1];
        c[k] = __ldg(cp + tv);
      }
#pragma unroll
      for (int k = 0; k < kTs; ++k) {
        const size_t tv = (size_t)(t + k) * cols;
        update(u[k], v[k], c[k]);
        o[2 * tv] = u[k];
        o[2 * tv + 1] = v[k];
      }
    }
    for (; t < T; ++t) {
      const size_t tv = (size_t)t * cols;
      float4 u = x[2 * tv], v = x[2 * tv + 1];
      update(u, v, __ldg(cp + tv));
      o[2 * tv] = u;
      o[2 * tv + 1] = v;
    }
  }
}

template <int FL>
static cudaError_t go_pass_col32(const Shape& s, const float* Xin, const float* C, const double* J_old,
                                 const double* J_cur, float* Rout, cudaStream_t st) {
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_pass_col32<FL>, 256, 0);
    return std::max(1, sms * std::max(per, 1));
  }();
  const int64_t cols = s.B * s.F;
  const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>((cols + 255) / 256, resident));
  k_pass_col32<FL><<<grid, 256, 0, st>>>(s.N, s.T, s.F, s.B, Xin, C, J_old, J_cur, Rout);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_pass(const Shape& s, int flags, const R* Xin, const R* C, const double* J_old,
                        const double* J_cur, R* Rout, R* stat_cost, R* stat_rho, int nchunk,
                        int tchunk, const LMState* lm, cudaStream_t st) {
#define SC_PASS(FL) \
  case FL:          \
    return go_pass<R, FL>(s, Xin, C, J_old, J_cur, Rout, stat_cost, stat_rho, nchunk, tchunk, lm, st);
  if constexpr (sizeof(R) == 4) {
    if (lm == nullptr && flags == (P_SUB | P_WRITE_R))
      return go_pass_col32<P_SUB | P_WRITE_R>(s, Xin, C, J_old, J_cur, Rout, st);
    if (lm == nullptr && flags == (P_OLD | P_SUB | P_WRITE_R))
      return go_pass_col32<P_OLD | P_SUB | P_WRITE_R>(s, Xin, C, J_old, J_cur, Rout, st);
  }
  switch (flags) {
    SC_PASS(P_SUB | P_STATS)                      // cost (and per-baseline sums) of a residual
    SC_PASS(P_SUB | P_WRITE_R | P_STATS)          // residual + cost
    SC_PASS(P_SUB | P_WRITE_R)                    // subtract one cluster's model
    SC_PASS(P_OLD | P_SUB | P_WRITE_R)            // replace one cluster's model
    default:
      return cudaErrorInvalidValue;
  }
#undef SC_PASS
}
template cudaError_t launch_pass<float>(const Shape&, int, const float*, const float*, const double*,
                                        const double*, float*, float*, float*, int, int,
                                        const LMState*, cudaStream_t);
template cudaError_t launch_pass<double>(const Shape&, int, const double*, const double*, const double*,
                                         const double*, double*, double*, double*, int, int,
                                         const LMState*, cudaStream_t);

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  return r;  // valid in thread 0
}

__global__ void k_sum_cost(const double* __restrict__ cpart, int N, double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) a += cpart[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) *out = a;
}

cudaError_t launch_sum_cost(const double* cpart, int N, double* out, cudaStream_t st) {
  k_sum_cost<<<1, 256, 0, st>>>(cpart, N, out);
  return cudaGetLastError();
}

template <typename R>
__global__ void k_sum_reals(const R* __restrict__ x, int64_t n, double* __restrict__ out) {
  __shared__ double sh[32];
  double a = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a += (double)x[i];
  a = block_sum(a, sh);
  if (threadIdx.x == 0) *out = a;
}

template <typename R>
cudaError_t launch_sum_reals(const R* x, int64_t n, double* out, cudaStream_t st) {
  k_sum_reals<R><<<1, 1024, 0, st>>>(x, n, out);
  return cudaGetLastError();
}
template cudaError_t launch_sum_reals<float>(const float*, int64_t, double*, cudaStream_t);
template cudaError_t launch_sum_reals<double>(const double*, int64_t, double*, cudaStream_t);

}  // namespace sc
