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
//
// Float64 arithmetic is slow on this GPU, so these kernels keep it to the
// sums and updates the method needs: the trial step spreads over several
// blocks (partial predicted decreases, summed in a fixed order by decide),
// maxima of magnitudes are taken on the bit patterns (integer compares),
// and the per-station maxima of |J^T r| come from the station sums.  In
// float32 the trial step also rounds the Jones once for the assembly of
// J^T J (Jf), so that no later kernel converts them per matrix element.
#include "sc_common.cuh"

namespace sc {

constexpr int kTrialThreads = 256;

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
// Maximum of non-negative doubles, compared as their bit patterns (the
// order of non-negative IEEE doubles is that of their bits).
__device__ __forceinline__ unsigned long long bred_umax(unsigned long long v, unsigned long long* sh) {
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sh[w] = v;
  __syncthreads();
  unsigned long long r = 0;
  for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = max(r, sh[i]);
  __syncthreads();
  return r;
}
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

__global__ void k_lm_init(LMState* lm, sc_lm_opts o, int N, LMBufs b, const double* __restrict__ J_src, size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  b = job_bufs(b, js, job);
  J_src = job_ptr(J_src, js, job);
  __shared__ double sh[32];
  __shared__ unsigned long long shu[32];
  double c = 0.0;
  unsigned long long dmax = 0, gmax = 0;
  for (int s = threadIdx.x; s < N; s += blockDim.x) {
    c += b.cp_cur[s];
    dmax = max(dmax, max(abs_bits(b.H_cur[4 * s]), abs_bits(b.H_cur[4 * s + 1])));
    gmax = max(gmax, abs_bits(b.gm_cur[s]));
  }
  for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) {
    const double v = J_src[k];
    if (J_src != b.J_cur) b.J_cur[k] = v;
    if (b.Jf_cur != nullptr) b.Jf_cur[k] = (float)v;
  }
  c = bred_sum(c, sh);
  dmax = bred_umax(dmax, shu);
  gmax = bred_umax(gmax, shu);
  if (threadIdx.x == 0) {
    lm->cost = c;
    lm->mu = o.tau * __longlong_as_double((long long)dmax);
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
    lm->done = (o.n_lm <= 0 || __longlong_as_double((long long)gmax) <= o.eps_grad * (1.0 + c)) ? 1 : 0;
  }
}

cudaError_t launch_lm_init(LMState* lm, const sc_lm_opts* o, int N, const LMBufs& b, const double* J_src,
                           cudaStream_t st, const Batch& bt) {
  k_lm_init<<<dim3(1, 1, bt.G), 512, 0, st>>>(lm, *o, N, b, J_src, bt.js);
  return cudaGetLastError();
}

// One thread per parameter: theta_trial = theta + d, and per block the
// partial predicted decrease sum d (mu d + g).
__global__ void __launch_bounds__(kTrialThreads) k_lm_trial(LMState* lm, int N, const double* __restrict__ x,
                                                          LMBufs b, size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm->done) return;
  b = job_bufs(b, js, job);
  x = job_ptr(x, js, job);
  __shared__ double sh[32];
  if (lm->notpd) {
    if (blockIdx.x == 0 && threadIdx.x == 0) lm->skip = 1;
    return;
  }
  const double mu = lm->mu;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  double pr = 0.0;
  if (k < 8 * N) {
    const double d = x[k];
    const double jt = b.J_cur[k] + d;
    b.J_trial[k] = jt;
    if (b.Jf_trial != nullptr) b.Jf_trial[k] = (float)jt;
    pr = d * (mu * d + b.g_cur[k]);
  }
  pr = bred_sum(pr, sh);
  if (threadIdx.x == 0) {
    b.pred_part[blockIdx.x] = pr;
    if (blockIdx.x == 0) lm->skip = 0;
  }
}

int lm_trial_blocks(int N) { return (8 * N + kTrialThreads - 1) / kTrialThreads; }

cudaError_t launch_lm_trial(LMState* lm, int N, const double* x, const LMBufs& b, cudaStream_t st,
                            const Batch& bt) {
  k_lm_trial<<<dim3(lm_trial_blocks(N), 1, bt.G), kTrialThreads, 0, st>>>(lm, N, x, b, bt.js);
  return cudaGetLastError();
}

__global__ void k_lm_decide(LMState* lm, int N, int n_pred, LMBufs b, size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm->done) return;
  b = job_bufs(b, js, job);
  __shared__ double sh[32];
  __shared__ unsigned long long shu[32];
  __shared__ int s_accept;
  const bool skipped = lm->skip != 0;
  double ct = 0.0;
  if (!skipped)
    for (int s = threadIdx.x; s < N; s += blockDim.x) ct += b.cp_trial[s];
  ct = bred_sum(ct, sh);
  if (threadIdx.x == 0) {
    double pred = 0.0;
    for (int i = 0; i < n_pred; ++i) pred += b.pred_part[i];
    double rho = -1.0;
    if (!skipped && pred > 0.0) rho = (lm->cost - ct) / pred;
    lm->pred = skipped ? 0.0 : pred;
    lm->rho = rho;
    lm->cost_trial = ct;
    s_accept = (!skipped && rho > 0.0) ? 1 : 0;
  }
  __syncthreads();
  const int acc = s_accept;
  if (acc) {
    for (int k = threadIdx.x; k < 8 * N; k += blockDim.x) {
      b.J_cur[k] = b.J_trial[k];
      b.g_cur[k] = b.g_trial[k];
      if (b.Jf_cur != nullptr) b.Jf_cur[k] = b.Jf_trial[k];
    }
    for (int k = threadIdx.x; k < 4 * N; k += blockDim.x) b.H_cur[k] = b.H_trial[k];
    for (int s = threadIdx.x; s < N; s += blockDim.x) b.gm_cur[s] = b.gm_trial[s];
  }
  // the gradient maximum of the state kept: the trial's when accepted
  const double* gm = acc ? b.gm_trial : b.gm_cur;
  unsigned long long gmax = 0;
  for (int s = threadIdx.x; s < N; s += blockDim.x) gmax = max(gmax, abs_bits(gm[s]));
  gmax = bred_umax(gmax, shu);
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
    if (lm->iter >= lm->n_lm || __longlong_as_double((long long)gmax) <= lm->eps_grad * (1.0 + lm->cost))
      lm->done = 1;
  }
}

cudaError_t launch_lm_decide(LMState* lm, int N, const LMBufs& b, cudaStream_t st, const Batch& bt) {
  k_lm_decide<<<dim3(1, 1, bt.G), 512, 0, st>>>(lm, N, lm_trial_blocks(N), b, bt.js);
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
