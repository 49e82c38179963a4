// Consensus across sub-bands: the steps of scaled-form consensus ADMM
// (Boyd et al. 2011, §7.1) that couple the sub-band calibrations through a
// smooth frequency model of the Jones, J_f ~ sum_p basis[f][p] Z_p.  The
// J-step is each band's SAGE run with a quadratic penalty (the station
// reduction of lm_pass.cu); these kernels do the rest:
//
//   fit     Z = (B^T B)^-1 B^T (J + U), per cluster and real parameter
//   target  a_f = basis[f] Z - U_f, the penalty target of band f's J-step
//   dual    U_f += J_f - basis[f] Z
//
// SAGECal distributes sub-bands over compute nodes (paper §1, §2); here
// they share one GPU.  Every array is float64: Jones and duals
// [n_bands][K][P], Z [K][n_poly][P] with P = 8N real parameters per cluster.
#include "sc_common.cuh"

namespace sc {

constexpr int kConsThreads = 256;

__global__ void __launch_bounds__(kConsThreads) k_consensus_fit(int n_bands, int n_poly, int K, int P,
                                                                const double* __restrict__ basis,
                                                                const double* __restrict__ J,
                                                                const double* __restrict__ U,
                                                                double* __restrict__ Z,
                                                                uint32_t* __restrict__ status) {
  __shared__ double G[kMaxPoly][2 * kMaxPoly];  // [B^T B | I], reduced to [I | (B^T B)^-1]
  __shared__ double W[kMaxPoly][kMaxBands];     // (B^T B)^-1 B^T
  __shared__ int s_ok;
  const int tid = threadIdx.x;
  for (int e = tid; e < n_poly * n_poly; e += blockDim.x) {
    const int r = e / n_poly, c = e - r * n_poly;
    double g = 0.0;
    for (int f = 0; f < n_bands; ++f) g += basis[f * n_poly + r] * basis[f * n_poly + c];
    G[r][c] = g;
    G[r][n_poly + c] = r == c ? 1.0 : 0.0;
  }
  __syncthreads();
  if (tid == 0) {
    // Gauss-Jordan elimination with partial pivoting
    double scale = 0.0;
    for (int r = 0; r < n_poly; ++r)
      for (int c = 0; c < n_poly; ++c) scale = fmax(scale, fabs(G[r][c]));
    int ok = scale > 0.0;
    for (int col = 0; col < n_poly && ok; ++col) {
      int piv = col;
      for (int r = col + 1; r < n_poly; ++r)
        if (fabs(G[r][col]) > fabs(G[piv][col])) piv = r;
      if (!(fabs(G[piv][col]) > 1e-14 * scale)) {
        ok = 0;
        break;
      }
      if (piv != col)
        for (int c = 0; c < 2 * n_poly; ++c) {
          const double t = G[col][c];
          G[col][c] = G[piv][c];
          G[piv][c] = t;
        }
      const double inv = 1.0 / G[col][col];
      for (int c = 0; c < 2 * n_poly; ++c) G[col][c] *= inv;
      for (int r = 0; r < n_poly; ++r) {
        if (r == col) continue;
        const double m = G[r][col];
        if (m != 0.0)
          for (int c = 0; c < 2 * n_poly; ++c) G[r][c] -= m * G[col][c];
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + tid;
  const int k = blockIdx.y;
  if (!s_ok) {  // the same for the whole block
    if (i < P)
      for (int p = 0; p < n_poly; ++p) Z[((size_t)k * n_poly + p) * P + i] = 0.0;
    if (i == 0 && k == 0) atomicOr(status, SC_STATUS_BASIS);
    return;
  }
  for (int e = tid; e < n_poly * n_bands; e += blockDim.x) {
    const int p = e / n_bands, f = e - p * n_bands;
    double w = 0.0;
    for (int l = 0; l < n_poly; ++l) w += G[p][n_poly + l] * basis[f * n_poly + l];
    W[p][f] = w;
  }
  __syncthreads();
  if (i >= P) return;
  double z[kMaxPoly];
#pragma unroll
  for (int p = 0; p < kMaxPoly; ++p) z[p] = 0.0;
  for (int f = 0; f < n_bands; ++f) {
    const size_t o = ((size_t)f * K + k) * P + i;
    const double y = J[o] + U[o];
#pragma unroll
    for (int p = 0; p < kMaxPoly; ++p)
      if (p < n_poly) z[p] += W[p][f] * y;
  }
#pragma unroll
  for (int p = 0; p < kMaxPoly; ++p)
    if (p < n_poly) Z[((size_t)k * n_poly + p) * P + i] = z[p];
}

// basis[f] Z for cluster k, parameter i
__device__ __forceinline__ double model_at(const double* __restrict__ basis, const double* __restrict__ Z,
                                           int f, int n_poly, int k, int P, int i) {
  double m = 0.0;
  for (int p = 0; p < n_poly; ++p) m += basis[f * n_poly + p] * Z[((size_t)k * n_poly + p) * P + i];
  return m;
}

__global__ void k_consensus_target(int band, int n_poly, int K, int P, const double* __restrict__ basis,
                                   const double* __restrict__ Z, const double* __restrict__ U,
                                   double* __restrict__ target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= P) return;
  target[(size_t)k * P + i] = model_at(basis, Z, band, n_poly, k, P, i) - U[((size_t)band * K + k) * P + i];
}

__global__ void k_consensus_dual(int n_poly, int K, int P, const double* __restrict__ basis,
                                 const double* __restrict__ J, const double* __restrict__ Z,
                                 double* __restrict__ U) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y, f = blockIdx.z;
  if (i >= P) return;
  const size_t o = ((size_t)f * K + k) * P + i;
  U[o] += J[o] - model_at(basis, Z, f, n_poly, k, P, i);
}

cudaError_t launch_consensus_fit(int n_bands, int n_poly, int K, int P, const double* basis,
                                 const double* J, const double* U, double* Z, uint32_t* status,
                                 cudaStream_t st) {
  dim3 grd((P + kConsThreads - 1) / kConsThreads, K);
  k_consensus_fit<<<grd, kConsThreads, 0, st>>>(n_bands, n_poly, K, P, basis, J, U, Z, status);
  return cudaGetLastError();
}

cudaError_t launch_consensus_target(int band, int n_poly, int K, int P, const double* basis,
                                    const double* Z, const double* U, double* target, cudaStream_t st) {
  dim3 grd((P + kConsThreads - 1) / kConsThreads, K);
  k_consensus_target<<<grd, kConsThreads, 0, st>>>(band, n_poly, K, P, basis, Z, U, target);
  return cudaGetLastError();
}

cudaError_t launch_consensus_dual(int n_bands, int n_poly, int K, int P, const double* basis,
                                  const double* J, const double* Z, double* U, cudaStream_t st) {
  dim3 grd((P + kConsThreads - 1) / kConsThreads, K, n_bands);
  k_consensus_dual<<<grd, kConsThreads, 0, st>>>(n_poly, K, P, basis, J, Z, U);
  return cudaGetLastError();
}

// Adds the device status word of a band workspace to the call's.
__global__ void k_or_status(const uint32_t* __restrict__ src, uint32_t* __restrict__ dst) {
  if (threadIdx.x == 0 && *src != 0) atomicOr(dst, *src);
}

cudaError_t launch_or_status(const uint32_t* src, uint32_t* dst, cudaStream_t st) {
  k_or_status<<<1, 32, 0, st>>>(src, dst);
  return cudaGetLastError();
}

}  // namespace sc
