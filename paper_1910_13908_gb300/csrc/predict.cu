// Step (a): point-source coherency prediction.
//
// C_pq(t,f) = sum_s S_s(f) exp(-2 pi i f/c (u l_s + v m_s + w (n_s - 1))), the
// coherency of a cluster of unpolarised point sources (SAGECal's sky model,
// one cluster = one calibration direction, paper §2).
//
// Mixed path: the (u,v,w) of baseline pq is uvw_p - uvw_q, so the phasor of a
// baseline is the product of two station phasors, e_p conj(e_q).  One kernel
// forms e_p(t,f,s) from a float64 argument reduced to [-1/2, 1/2] turns before
// a float32 sincospi (N phasors per (t,f,s) instead of B), the other contracts
// them, C_pq = sum_s (S_s e_p,s) conj(e_q,s), with 64x64 station tiles in
// shared memory and float32 accumulation.  It also sums w_pq = sum |C_pq|^2
// over (t,f), the only data the Gauss-Newton matrix needs.
//
// Plain FP64 path: every (source, baseline, timeslot, channel) phase and
// sincos in float64, one thread per (t, b).
#include "sc_common.cuh"

namespace sc {

__device__ __forceinline__ double n_minus_1(double l, double m) {
  double r2 = l * l + m * m;
  return -r2 / (1.0 + sqrt(1.0 - r2));
}

// E[(tf * S + s) * N + p] = exp(-2 pi i f/c uvw_p . (l, m, n-1)), Sf[f*S + s] = S_s(f)
__global__ void k_station_phasors(int N, int T, int F, int S, const double* __restrict__ uvw,
                                  const double* __restrict__ freqs, const double* __restrict__ l,
                                  const double* __restrict__ m, const double* __restrict__ flux,
                                  const double* __restrict__ alpha, double f0,
                                  float2* __restrict__ E, float* __restrict__ Sf) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  int s = blockIdx.y;
  int tf = blockIdx.z;
  int t = tf / F, f = tf % F;
  double fr = freqs[f];
  if (p == 0 && t == 0) Sf[f * S + s] = (float)(flux[s] * pow(fr / f0, alpha[s]));
  if (p >= N) return;
  double ls = l[s], ms = m[s];
  double nm1 = n_minus_1(ls, ms);
  const double* x = uvw + ((size_t)t * N + p) * 3;
  double path = fma(x[0], ls, fma(x[1], ms, x[2] * nm1));  // metres
  double turns = path * (fr / kCLight);
  float y = (float)(turns - rint(turns));                  // [-1/2, 1/2] turns
  float sn, cs;
  sincospif(2.0f * y, &sn, &cs);
  E[((size_t)tf * S + s) * N + p] = make_float2(cs, -sn);
}

cudaError_t launch_station_phasors(const Shape& s, const double* uvw, const double* freqs,
                                   const double* l, const double* m, const double* flux,
                                   const double* alpha, double f0, int S, float2* E, float* Sf,
                                   cudaStream_t st) {
  if (S <= 0) return cudaSuccess;
  dim3 blk(128);
  dim3 grd((s.N + 127) / 128, S, s.T * s.F);
  k_station_phasors<<<grd, blk, 0, st>>>(s.N, s.T, s.F, S, uvw, freqs, l, m, flux, alpha, f0, E, Sf);
  return cudaGetLastError();
}

// ---- float32 contraction over sources --------------------------------------------------------

constexpr int kCT = 64;   // stations per tile edge
constexpr int kCS = 32;   // sources staged per step

__global__ void __launch_bounds__(256) k_coherency_f32(int N, int T, int F, int S, int64_t B, int nt,
                                                        int splits, const float2* __restrict__ E,
                                                        const float* __restrict__ Sf,
                                                        float2* __restrict__ C,
                                                        float* __restrict__ wpart) {
  __shared__ float2 sa[kCS][kCT];  // S_s(f) e_p,s
  __shared__ float2 se[kCS][kCT];  // e_q,s
  // tile (tp, tq), tp <= tq, from the linear block index
  int L = blockIdx.x, tp = 0;
  while (L >= nt - tp) { L -= nt - tp; ++tp; }
  int tq = tp + L;
  int p0 = tp * kCT, q0 = tq * kCT;
  int split = blockIdx.y;
  int TF = T * F;
  int tf0 = (int)((int64_t)TF * split / splits), tf1 = (int)((int64_t)TF * (split + 1) / splits);
  int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  float wacc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) wacc[i][j] = 0.f;

  for (int tf = tf0; tf < tf1; ++tf) {
    int t = tf / F, f = tf % F;
    float ar[4][4], ai[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) ar[i][j] = ai[i][j] = 0.f;
    const float2* Et = E + (size_t)tf * S * N;
    for (int s0 = 0; s0 < S; s0 += kCS) {
      // stage kCS sources x 64 stations of each side
      for (int e = threadIdx.x; e < kCS * kCT; e += blockDim.x) {
        int ss = e / kCT, c = e % kCT;
        int sidx = s0 + ss;
        float2 va = make_float2(0.f, 0.f), ve = make_float2(0.f, 0.f);
        if (sidx < S) {
          if (p0 + c < N) {
            float2 v = Et[(size_t)sidx * N + p0 + c];
            float fl = Sf[f * S + sidx];
            va = make_float2(v.x * fl, v.y * fl);
          }
          if (q0 + c < N) ve = Et[(size_t)sidx * N + q0 + c];
        }
        sa[ss][c] = va;
        se[ss][c] = ve;
      }
      __syncthreads();
      int ns = min(kCS, S - s0);
      for (int ss = 0; ss < ns; ++ss) {
        float2 a[4], e[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = sa[ss][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) e[j] = se[ss][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            // a * conj(e)
            ar[i][j] = fmaf(a[i].x, e[j].x, fmaf(a[i].y, e[j].y, ar[i][j]));
            ai[i][j] = fmaf(a[i].y, e[j].x, fmaf(-a[i].x, e[j].y, ai[i][j]));
          }
      }
      __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      int p = p0 + ty + 16 * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        int q = q0 + tx + 16 * j;
        if (p < q && q < N) {
          int64_t b = bl_index(p, q, N);
          C[((size_t)t * B + b) * F + f] = make_float2(ar[i][j], ai[i][j]);
          wacc[i][j] += ar[i][j] * ar[i][j] + ai[i][j] * ai[i][j];
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int q = q0 + tx + 16 * j;
      if (p < q && q < N) wpart[(size_t)split * B + bl_index(p, q, N)] = wacc[i][j];
    }
  }
}

cudaError_t launch_coherency_f32(const Shape& s, int S, const float2* E, const float* Sf,
                                 float2* C, float* wpart, int splits, cudaStream_t st) {
  int nt = (s.N + kCT - 1) / kCT;
  int tiles = nt * (nt + 1) / 2;
  dim3 grd(tiles, splits);
  if (S <= 0) {
    // an empty cluster predicts zero coherencies
    cudaError_t e = cudaMemsetAsync(C, 0, sizeof(float2) * (size_t)s.T * s.B * s.F, st);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(wpart, 0, sizeof(float) * (size_t)splits * s.B, st);
  }
  k_coherency_f32<<<grd, 256, 0, st>>>(s.N, s.T, s.F, S, s.B, nt, splits, E, Sf, C, wpart);
  return cudaGetLastError();
}

__global__ void k_sum_parts(const float* __restrict__ part, int splits, int64_t B, float* __restrict__ w) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float acc = 0.f;
  for (int i = 0; i < splits; ++i) acc += part[(size_t)i * B + b];
  w[b] = acc;
}

cudaError_t launch_sum_parts(const float* wpart, int splits, int64_t B, float* w, cudaStream_t st) {
  k_sum_parts<<<(unsigned)((B + 255) / 256), 256, 0, st>>>(wpart, splits, B, w);
  return cudaGetLastError();
}

// ---- plain float64 path --------------------------------------------------------------------

__global__ void k_predict_f64(int N, int T, int F, int S, int64_t B, const double* __restrict__ uvw,
                              const double* __restrict__ freqs, const double* __restrict__ l,
                              const double* __restrict__ m, const double* __restrict__ flux,
                              const double* __restrict__ alpha, double f0, double2* __restrict__ C) {
  int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)T * B) return;
  int t = (int)(idx / B);
  int64_t b = idx % B;
  int p, q;
  bl_pair(b, N, p, q);
  const double* xp = uvw + ((size_t)t * N + p) * 3;
  const double* xq = uvw + ((size_t)t * N + q) * 3;
  double u = xp[0] - xq[0], v = xp[1] - xq[1], w = xp[2] - xq[2];
  for (int f = 0; f < F; ++f) {
    double fr = freqs[f];
    double re = 0.0, im = 0.0;
    for (int s = 0; s < S; ++s) {
      double ls = __ldg(l + s), ms = __ldg(m + s);
      double path = u * ls + v * ms + w * n_minus_1(ls, ms);
      double turns = path * (fr / kCLight);
      double sn, cs;
      sincospi(2.0 * (turns - rint(turns)), &sn, &cs);
      double S_f = __ldg(flux + s) * pow(fr / f0, __ldg(alpha + s));
      re += S_f * cs;
      im -= S_f * sn;
    }
    C[((size_t)t * B + b) * F + f] = make_double2(re, im);
  }
}

cudaError_t launch_predict_f64(const Shape& s, const double* uvw, const double* freqs,
                               const double* l, const double* m, const double* flux,
                               const double* alpha, double f0, int S, double2* C,
                               cudaStream_t st) {
  int64_t n = (int64_t)s.T * s.B;
  k_predict_f64<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(s.N, s.T, s.F, S, s.B, uvw, freqs, l, m,
                                                              flux, alpha, f0, C);
  return cudaGetLastError();
}

// w_pq = sum_{t,f} |C_pq(t,f)|^2
template <typename R>
__global__ void k_w_from_C(int T, int F, int64_t B, const R* __restrict__ C, R* __restrict__ w) {
  int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  R acc = 0;
  for (int t = 0; t < T; ++t)
    for (int f = 0; f < F; ++f) {
      cx<R> c = ld_c(C + 2 * (((size_t)t * B + b) * F + f));
      acc += norm2(c);
    }
  w[b] = acc;
}

template <typename R>
cudaError_t launch_w_from_C(const Shape& s, const R* C, R* w, cudaStream_t st) {
  k_w_from_C<R><<<(unsigned)((s.B + 255) / 256), 256, 0, st>>>(s.T, s.F, s.B, C, w);
  return cudaGetLastError();
}
template cudaError_t launch_w_from_C<float>(const Shape&, const float*, float*, cudaStream_t);
template cudaError_t launch_w_from_C<double>(const Shape&, const double*, double*, cudaStream_t);

}  // namespace sc
