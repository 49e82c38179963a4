// Prediction of polarised and Gaussian-extended sources: full 2x2 coherencies
//
//   C_pq(t,f) = sum_s (f/f0)^alpha_s G_s(u f/c, v f/c)
//               exp(-2 pi i f/c (u l_s + v m_s + w (n_s - 1))) B_s,
//   B_s = [[I + Q, U + iV], [U - iV, I - Q]],
//   G_s = exp(-2 pi^2 (sigma_a^2 u_a^2 + sigma_b^2 u_b^2)),
//
// with sigma = FWHM / (2 sqrt(2 ln 2)) and (u_a, u_b) the baseline projected
// on the major axis (sin pa, cos pa) and the minor axis (cos pa, -sin pa);
// G = 1 for a point source.  SAGECal's sky models carry full Stokes and
// Gaussian sources besides points (one cluster = one calibration direction,
// paper §2).
//
// Mixed path: the baseline phasor is the product of two station phasors
// (k_station_phasors, float64 argument reduced to [-1/2, 1/2] turns).  Per
// channel and source, k_source_params folds the spectral law into the four
// Stokes parameters and the shape into the quadratic form
// A u^2 + 2B uv + C v^2 of the baseline in metres, so the contraction needs no
// trigonometry: per (source, baseline) one complex product, for an extended
// source one expf, and four complex FMAs into the I, Q, U and V sums; B_s's
// layout is applied once per output.  32x32 station tiles, 2x2 pairs per
// thread, sources staged through shared memory.
//
// Plain FP64 path: everything per (source, baseline, timeslot, channel) in
// float64, one thread per (t, b).
#include "sc_common.cuh"

namespace sc {

namespace {
constexpr double kFwhmPerSigma = 2.3548200450309493;  // 2 sqrt(2 ln 2)
constexpr double kPi = 3.14159265358979323846;

__device__ __forceinline__ double nm1_full(double l, double m) {
  double r2 = l * l + m * m;
  return -r2 / (1.0 + sqrt(1.0 - r2));
}

// Coefficients (A, 2B, C) of the Gaussian exponent in the baseline's metres
// at frequency fr: exponent = A u^2 + 2B u v + C v^2.
__device__ __forceinline__ void gauss_form(double maj, double mnr, double pa, double fr, double& A,
                                           double& B2, double& C) {
  const double sa = maj / kFwhmPerSigma, sb = mnr / kFwhmPerSigma;
  const double k = 2.0 * kPi * kPi * (fr / kCLight) * (fr / kCLight);
  double sp, cp;
  sincos(pa, &sp, &cp);
  const double a2 = sa * sa, b2 = sb * sb;
  A = k * (a2 * sp * sp + b2 * cp * cp);
  B2 = k * 2.0 * (a2 - b2) * sp * cp;
  C = k * (a2 * cp * cp + b2 * sp * sp);
}
}  // namespace

// st[f*S + s] = (I, Q, U, V)_s (f/f0)^alpha_s; gq[f*S + s] = (A, 2B, C, extended)
__global__ void k_source_params(int F, int S, const double* __restrict__ freqs,
                                const double* __restrict__ I, const double* __restrict__ Q,
                                const double* __restrict__ U, const double* __restrict__ V,
                                const double* __restrict__ alpha, const double* __restrict__ maj,
                                const double* __restrict__ mnr, const double* __restrict__ pa, double f0,
                                float4* __restrict__ st, float4* __restrict__ gq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F * S) return;
  const int f = i / S, s = i - f * S;
  const double fr = freqs[f];
  const double sp = pow(fr / f0, alpha[s]);
  st[i] = make_float4((float)(I[s] * sp), (float)(Q[s] * sp), (float)(U[s] * sp), (float)(V[s] * sp));
  double A, B2, C;
  gauss_form(maj[s], mnr[s], pa[s], fr, A, B2, C);
  const bool ext = maj[s] != 0.0 || mnr[s] != 0.0;
  gq[i] = make_float4((float)A, (float)B2, (float)C, ext ? 1.f : 0.f);
}

constexpr int kFT = 32;  // stations per tile edge
constexpr int kFS = 32;  // sources staged per step

__global__ void __launch_bounds__(256) k_coherency_full_f32(int N, int T, int F, int S, int64_t B, int nt,
                                                             const double* __restrict__ uvw,
                                                             const float2* __restrict__ E,
                                                             const float4* __restrict__ st,
                                                             const float4* __restrict__ gq,
                                                             float* __restrict__ C) {
  __shared__ float2 sp_[kFS][kFT];  // e_p,s
  __shared__ float2 sq_[kFS][kFT];  // e_q,s
  __shared__ float4 sst[kFS];
  __shared__ float4 sgq[kFS];
  int L = blockIdx.x, tp = 0;
  while (L >= nt - tp) {
    L -= nt - tp;
    ++tp;
  }
  const int tq = tp + L;
  const int p0 = tp * kFT, q0 = tq * kFT;
  const int tf = blockIdx.y;
  const int t = tf / F, f = tf - t * F;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;

  // baseline (u, v) in metres of the thread's 2x2 pairs
  float bu[2][2], bv[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int p = min(p0 + ty + 16 * i, N - 1), q = min(q0 + tx + 16 * j, N - 1);
      const double* xp = uvw + ((size_t)t * N + p) * 3;
      const double* xq = uvw + ((size_t)t * N + q) * 3;
      bu[i][j] = (float)(xp[0] - xq[0]);
      bv[i][j] = (float)(xp[1] - xq[1]);
    }
  float2 aI[2][2], aQ[2][2], aU[2][2], aV[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) aI[i][j] = aQ[i][j] = aU[i][j] = aV[i][j] = make_float2(0.f, 0.f);

  const float2* Et = E + (size_t)tf * S * N;
  for (int s0 = 0; s0 < S; s0 += kFS) {
    for (int e = threadIdx.x; e < kFS * kFT; e += blockDim.x) {
      const int ss = e / kFT, c = e % kFT;
      const int sidx = s0 + ss;
      float2 va = make_float2(0.f, 0.f), ve = make_float2(0.f, 0.f);
      if (sidx < S) {
        if (p0 + c < N) va = Et[(size_t)sidx * N + p0 + c];
        if (q0 + c < N) ve = Et[(size_t)sidx * N + q0 + c];
      }
      sp_[ss][c] = va;
      sq_[ss][c] = ve;
    }
    if (threadIdx.x < kFS) {
      const int sidx = s0 + threadIdx.x;
      sst[threadIdx.x] = sidx < S ? st[(size_t)f * S + sidx] : make_float4(0.f, 0.f, 0.f, 0.f);
      sgq[threadIdx.x] = sidx < S ? gq[(size_t)f * S + sidx] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    const int ns = min(kFS, S - s0);
    for (int ss = 0; ss < ns; ++ss) {
      const float4 k4 = sst[ss];
      const float4 g4 = sgq[ss];
      float2 a[2], e[2];
#pragma unroll
      for (int i = 0; i < 2; ++i) a[i] = sp_[ss][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 2; ++j) e[j] = sq_[ss][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          // a * conj(e)
          float pr = fmaf(a[i].x, e[j].x, a[i].y * e[j].y);
          float pi = fmaf(a[i].y, e[j].x, -a[i].x * e[j].y);
          if (g4.w != 0.f) {  // the same branch for the whole block
            const float u = bu[i][j], v = bv[i][j];
            const float x = fmaf(g4.x * u, u, fmaf(g4.y * u, v, g4.z * v * v));
            const float att = expf(-x);
            pr *= att;
            pi *= att;
          }
          aI[i][j].x = fmaf(pr, k4.x, aI[i][j].x);
          aI[i][j].y = fmaf(pi, k4.x, aI[i][j].y);
          aQ[i][j].x = fmaf(pr, k4.y, aQ[i][j].x);
          aQ[i][j].y = fmaf(pi, k4.y, aQ[i][j].y);
          aU[i][j].x = fmaf(pr, k4.z, aU[i][j].x);
          aU[i][j].y = fmaf(pi, k4.z, aU[i][j].y);
          aV[i][j].x = fmaf(pr, k4.w, aV[i][j].x);
          aV[i][j].y = fmaf(pi, k4.w, aV[i][j].y);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int p = p0 + ty + 16 * i;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int q = q0 + tx + 16 * j;
      if (p < q && q < N) {
        const int64_t b = bl_index(p, q, N);
        const float2 cI = aI[i][j], cQ = aQ[i][j], cU = aU[i][j], cV = aV[i][j];
        float4* out = reinterpret_cast<float4*>(C + 8 * (((size_t)t * B + b) * F + f));
        // XX = I + Q, XY = U + iV, YX = U - iV, YY = I - Q
        out[0] = make_float4(cI.x + cQ.x, cI.y + cQ.y, cU.x - cV.y, cU.y + cV.x);
        out[1] = make_float4(cU.x + cV.y, cU.y - cV.x, cI.x - cQ.x, cI.y - cQ.y);
      }
    }
  }
}

// ---- plain float64 path --------------------------------------------------------------------

__global__ void k_predict_full_f64(int N, int T, int F, int S, int64_t B, const double* __restrict__ uvw,
                                   const double* __restrict__ freqs, const double* __restrict__ l,
                                   const double* __restrict__ m, const double* __restrict__ I,
                                   const double* __restrict__ Q, const double* __restrict__ U,
                                   const double* __restrict__ V, const double* __restrict__ alpha,
                                   const double* __restrict__ maj, const double* __restrict__ mnr,
                                   const double* __restrict__ pa, double f0, double* __restrict__ C) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (int64_t)T * B) return;
  const int t = (int)(idx / B);
  const int64_t b = idx % B;
  int p, q;
  bl_pair(b, N, p, q);
  const double* xp = uvw + ((size_t)t * N + p) * 3;
  const double* xq = uvw + ((size_t)t * N + q) * 3;
  const double u = xp[0] - xq[0], v = xp[1] - xq[1], w = xp[2] - xq[2];
  for (int f = 0; f < F; ++f) {
    const double fr = freqs[f];
    double2 cI = make_double2(0, 0), cQ = cI, cU = cI, cV = cI;
    for (int s = 0; s < S; ++s) {
      const double ls = __ldg(l + s), ms = __ldg(m + s);
      const double path = u * ls + v * ms + w * nm1_full(ls, ms);
      const double turns = path * (fr / kCLight);
      double sn, cs;
      sincospi(2.0 * (turns - rint(turns)), &sn, &cs);
      double amp = pow(fr / f0, __ldg(alpha + s));
      const double a_maj = __ldg(maj + s), a_mnr = __ldg(mnr + s);
      if (a_maj != 0.0 || a_mnr != 0.0) {
        double A, B2, Cq;
        gauss_form(a_maj, a_mnr, __ldg(pa + s), fr, A, B2, Cq);
        amp *= exp(-(A * u * u + B2 * u * v + Cq * v * v));
      }
      const double pr = amp * cs, pi = -amp * sn;
      const double si = __ldg(I + s), sq = __ldg(Q + s), su = __ldg(U + s), sv = __ldg(V + s);
      cI.x += pr * si; cI.y += pi * si;
      cQ.x += pr * sq; cQ.y += pi * sq;
      cU.x += pr * su; cU.y += pi * su;
      cV.x += pr * sv; cV.y += pi * sv;
    }
    double2* out = reinterpret_cast<double2*>(C + 8 * (((size_t)t * B + b) * F + f));
    out[0] = make_double2(cI.x + cQ.x, cI.y + cQ.y);
    out[1] = make_double2(cU.x - cV.y, cU.y + cV.x);
    out[2] = make_double2(cU.x + cV.y, cU.y - cV.x);
    out[3] = make_double2(cI.x - cQ.x, cI.y - cQ.y);
  }
}

// ---- launchers -------------------------------------------------------------------------------

cudaError_t launch_source_params(const Shape& s, int S, const double* freqs, const SkyFull& k, float4* st,
                                 float4* gq, cudaStream_t stream) {
  if (S <= 0) return cudaSuccess;
  const int n = s.F * S;
  k_source_params<<<(n + 127) / 128, 128, 0, stream>>>(s.F, S, freqs, k.I, k.Q, k.U, k.V, k.alpha, k.maj,
                                                       k.mnr, k.pa, k.f0, st, gq);
  return cudaGetLastError();
}

cudaError_t launch_coherency_full_f32(const Shape& s, int S, const double* uvw, const float2* E,
                                      const float4* st, const float4* gq, float* C, cudaStream_t stream) {
  if (S <= 0) return cudaMemsetAsync(C, 0, sizeof(float) * 8 * (size_t)s.T * s.B * s.F, stream);
  const int nt = (s.N + kFT - 1) / kFT;
  dim3 grd(nt * (nt + 1) / 2, s.T * s.F);
  k_coherency_full_f32<<<grd, 256, 0, stream>>>(s.N, s.T, s.F, S, s.B, nt, uvw, E, st, gq, C);
  return cudaGetLastError();
}

cudaError_t launch_predict_full_f64(const Shape& s, int S, const double* uvw, const double* freqs,
                                    const SkyFull& k, double* C, cudaStream_t stream) {
  if (S <= 0) return cudaMemsetAsync(C, 0, sizeof(double) * 8 * (size_t)s.T * s.B * s.F, stream);
  const int64_t n = (int64_t)s.T * s.B;
  k_predict_full_f64<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(
      s.N, s.T, s.F, S, s.B, uvw, freqs, k.l, k.m, k.I, k.Q, k.U, k.V, k.alpha, k.maj, k.mnr, k.pa, k.f0, C);
  return cudaGetLastError();
}

}  // namespace sc
