// Levenberg-Marquardt control on the device (Madsen, Nielsen & Tingleff 2004,
// Alg. 3.16: the step solves (J^T J + mu I) d = J^T r), so that a whole
// solve is a fixed sequence of launches with no host round trip:
//   init:   cost = sum of station partial costs, mu = tau max diag(J^T J),
//           nu = 2, stop if max|J^T r| <= eps (1 + cost)
//   trial:  theta_trial = theta + d, predicted decrease d^T (mu d + g)
//   decide: rho = (cost - cost_trial) / predicted; rho > 0 accepts the step
//           (mu *= max(1/3, 1 - (2 rho - 1)^3), nu = 2), otherwise
//           mu *= nu, nu *= 2; a non-positive-definite factorisation counts
//           as a rejection.  Every later kernel of the solve returns at once
//           after the last iteration or the gradient stop.
#include "sc_common.cuh"

namespace sc {

__device__ __forceinline__ double bred_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += sh[i];
  __syncthreads();
  return r;  // valid in every thread
}
__device__ __forceinline__ double bred_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmax(r, sh[i]);
  __syncthreads();
  return r;
}

__global__ void k_lm_init(LMState* lm, sc_lm_opts o, int N, const double* __restrict__ H,
                          const double* __restrict__ g, const double* __restrict__ cpart,
                          const double* __restrict__ J_src, double* __restrict__ J_cur) {
  __shared__ double sh[32];
  double c = 0.0, dmax = 0.0, gmax = 0.0;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    c += cpart[s];
    dmax = fmax(dmax, fmax(H[4 * s], H[4 * s + 1]));
  }
  for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) {
    gmax = fmax(gmax, fabs(g[k]));
    if (J_src != J_cur) J_cur[k] = J_src[k];
  }
  c = bred_sum(c, sh);
  dmax = bred_max(dmax, sh);
  gmax = bred_max(gmax, sh);
  if (threadIdx.x == 0) {
    lm->cost = c;
    lm->mu = o.tau * dmax;
    lm->nu = 2.0;
    lm->lm_tau = o.tau;
    lm->eps_grad = o.eps_grad;
    lm->iter = 0;
    lm->n_lm = o.n_lm;
    lm->notpd = 0;
    lm->skip = 0;
    lm->accepted = 0;
    lm->rho = 0.0;
    lm->pred = 0.0;
    lm->cost_trial = 0.0;
    lm->done = (o.n_lm <= 0 || gmax <= o.eps_grad * (1.0 + c)) ? 1 : 0;
  }
}

cudaError_t launch_lm_init(LMState* lm, const sc_lm_opts* o, int N, const double* H,
                           const double* g, const double* cpart, const double* J_src,
                           double* J_cur, cudaStream_t st) {
  k_lm_init<<<1, 256, 0, st>>>(lm, *o, N, H, g, cpart, J_src, J_cur);
  return cudaGetLastError();
}

__global__ void k_lm_trial(LMState* lm, int N, const double* __restrict__ J_cur,
                           const double* __restrict__ x, const double* __restrict__ H,
                           const double* __restrict__ g, double* __restrict__ J_trial) {
  if (lm->done) return;
  __shared__ double sh[32];
  if (lm->notpd) {
    if (threadIdx.x == 0) lm->skip = 1;
    return;
  }
  double mu = lm->mu, pr = 0.0;
  for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) {
    double d = x[k];
    J_trial[k] = J_cur[k] + d;
    pr += d * (mu * d + g[k]);
  }
  pr = bred_sum(pr, sh);
  if (threadIdx.x == 0) {
    lm->pred = pr;
    lm->skip = 0;
  }
}

cudaError_t launch_lm_trial(LMState* lm, int N, int Ppad, const double* J_cur, const double* x,
                            const double* H, const double* g, double* J_trial, cudaStream_t st) {
  (void)Ppad;
  k_lm_trial<<<1, 1024, 0, st>>>(lm, N, J_cur, x, H, g, J_trial);
  return cudaGetLastError();
}

__global__ void k_lm_decide(LMState* lm, int N, const double* __restrict__ cpart_trial,
                            double* __restrict__ J_cur, const double* __restrict__ J_trial,
                            double* __restrict__ g_cur, const double* __restrict__ g_trial,
                            double* __restrict__ H_cur, const double* __restrict__ H_trial) {
  if (lm->done) return;
  __shared__ double sh[32];
  __shared__ int s_accept;
  bool skipped = lm->skip != 0;
  double ct = 0.0;
  if (!skipped)
    for (int s = threadIdx.x; s < N; s += blockDim.x) ct += cpart_trial[s];
  ct = bred_sum(ct, sh);
  if (threadIdx.x == 0) {
    double rho = -1.0;
    if (!skipped && lm->pred > 0.0) rho = (lm->cost - ct) / lm->pred;
    lm->rho = rho;
    lm->cost_trial = ct;
    s_accept = (!skipped && rho > 0.0) ? 1 : 0;
  }
  __syncthreads();
  int acc = s_accept;
  if (acc) {
    for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) {
      J_cur[k] = J_trial[k];
      g_cur[k] = g_trial[k];
    }
    for (int k = threadIdx.x; k < 4 * N; k += blockDim.x) H_cur[k] = H_trial[k];
  }
  __syncthreads();
  double gmax = 0.0;
  for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) gmax = fmax(gmax, fabs(g_cur[k]));
  gmax = bred_max(gmax, sh);
  if (threadIdx.x == 0) {
    if (acc) {
      double t = 2.0 * lm->rho - 1.0;
      lm->mu *= fmax(1.0 / 3.0, 1.0 - t * t * t);
      lm->nu = 2.0;
      lm->cost = ct;
      lm->accepted += 1;
    } else {
      lm->mu *= lm->nu;
      lm->nu *= 2.0;
    }
    lm->iter += 1;
    lm->notpd = 0;
    lm->skip = 0;
    if (lm->iter >= lm->n_lm || gmax <= lm->eps_grad * (1.0 + lm->cost)) lm->done = 1;
  }
}

cudaError_t launch_lm_decide(LMState* lm, int N, const double* cpart_trial, double* J_cur,
                             const double* J_trial, double* g_cur, const double* g_trial,
                             double* H_cur, const double* H_trial, cudaStream_t st) {
  k_lm_decide<<<1, 1024, 0, st>>>(lm, N, cpart_trial, J_cur, J_trial, g_cur, g_trial, H_cur, H_trial);
  return cudaGetLastError();
}

__global__ void k_lm_finish(const LMState* __restrict__ lm, const double* __restrict__ J_cur, int N,
                            double* __restrict__ J_out, double* __restrict__ cost_out,
                            int32_t* __restrict__ iters_out) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < 8 * N; k += gridDim.x * blockDim.x)
    J_out[k] = J_cur[k];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    if (cost_out) *cost_out = lm->cost;
    if (iters_out) *iters_out = lm->iter;
  }
}

cudaError_t launch_lm_finish(const LMState* lm, const double* J_cur, int N, double* J_out,
                             double* cost_out, int32_t* iters_out, cudaStream_t st) {
  k_lm_finish<<<(8 * N + 255) / 256, 256, 0, st>>>(lm, J_cur, N, J_out, cost_out, iters_out);
  return cudaGetLastError();
}

}  // namespace sc
