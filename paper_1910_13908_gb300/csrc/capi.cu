// The C ABI (include/sagecal_gb.h): argument checks, workspace layout, and the
// host-side sequencing of the kernels for one cluster solve and for a SAGE
// job.  Everything is enqueued on the caller's stream; no call synchronises,
// allocates or round-trips to the host between kernels.
#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstddef>
#include <string>
#include <thread>
#include <vector>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "sc_common.cuh"

namespace sc {

// ---- errors --------------------------------------------------------------------------------

static thread_local int g_err = SC_OK;
static thread_local char g_msg[512] = "";

static int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  g_err = code;
  return code;
}
static int ok() {
  g_err = SC_OK;
  g_msg[0] = 0;
  return SC_OK;
}

#define SC_CUDA(expr)                                                                      \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// one kernel launch of kind K on stream c.st, timed when profiling is on
#define SC_LAUNCH(K, expr)                                                                 \
  do {                                                                                     \
    prof_start(K, c.st);                                                                   \
    cudaError_t e_ = (expr);                                                               \
    prof_stop(K, c.st);                                                                    \
    if (e_ != cudaSuccess) return fail(SC_ECUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// ---- workspace layout ----------------------------------------------------------------------

static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// (timeslot, channel) splits of the point-source contraction: enough
// (station tile pair, split) blocks for two per multiprocessor.
static int coherency_splits(const Shape& s, int sms) {
  const int nt = (s.N + 63) / 64, tiles = nt * (nt + 1) / 2;
  return std::max(1, std::min(s.T * s.F, (2 * sms + tiles - 1) / tiles));
}

// Multiprocessors of the current device, looked up once per device.
static int device_sms() {
  constexpr int kDevs = 64;
  static std::atomic<int> cache[kDevs];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kDevs) return 1;
  int v = cache[dev].load(std::memory_order_relaxed);
  if (v > 0) return v;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 1;
  v = std::min(v, kMaxSMs);
  cache[dev].store(v, std::memory_order_relaxed);
  return v;
}

Workspace plan_workspace(const Shape& s, bool job) {
  Workspace L{};
  size_t rs = s.prec == SC_MIXED ? 4 : 8;
  size_t N = s.N, T = s.T, F = s.F, K = s.K, B = (size_t)s.B;
  size_t Smax = std::max(s.S_max, 1);
  L.Ppad = (int)((8 * N + kNB - 1) / kNB * kNB);
  L.nT = L.Ppad / kNB;
  // enough (baseline, timeslot-chunk) work items to fill the GPU several times
  const int64_t target = 1 << 18;
  int64_t tb = (int64_t)T * (int64_t)B;
  L.tchunk = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)T, tb / target));
  L.nchunk = (int)((T + L.tchunk - 1) / L.tchunk);
  // room for the predict kernel's (timeslot, channel) splits on a GPU of up
  // to kMaxSMs multiprocessors; the launch takes what the current device
  // needs (coherency_splits), so the size does not depend on the device
  L.splits = coherency_splits(s, kMaxSMs);
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + std::max<size_t>(bytes, 1));
    return at;
  };
  L.status = take(256);
  L.lm = take(sizeof(LMState));
  L.C = job ? take(K * T * B * F * 2 * rs) : 0;
  L.w = take((job ? K : 1) * B * rs);
  L.wpart = take((size_t)L.splits * B * 4);
  L.Rres = job ? take(T * B * F * 8 * rs) : 0;
  L.E = s.prec == SC_MIXED ? take(T * F * Smax * N * 8) : 0;
  L.Sf = take(F * Smax * 8);
  L.stat_cost = take((size_t)L.nchunk * B * rs);
  L.stat_rho = take((size_t)L.nchunk * B * 8 * rs);
  L.lstat = take(lm_stats_doubles(s.T, s.B) * 8);
  L.part = take(lm_part_doubles(s.N) * 8);
  L.J_old = take(8 * N * 8);
  L.J_cur = take(8 * N * 8);
  L.J_trial = take(8 * N * 8);
  L.g_cur = take(8 * N * 8);
  L.g_trial = take(8 * N * 8);
  L.H_cur = take(4 * N * 8);
  L.H_trial = take(4 * N * 8);
  L.cpart_cur = take(N * 8);
  L.cpart_trial = take(N * 8);
  L.gm_cur = take(N * 8);
  L.gm_trial = take(N * 8);
  L.pred_part = take((8 * N / 256 + 1) * 8);
  L.Jf_cur = take(8 * N * 4);
  L.Jf_trial = take(8 * N * 4);
  L.x = take((size_t)L.Ppad * 8);
  L.rvec = take((size_t)L.Ppad * 8);
  L.ry = take((size_t)L.Ppad * 8);
  L.bvec = take((size_t)L.Ppad * 2 * rs);
  L.A = take((size_t)L.Ppad * L.Ppad * rs);
  L.Linv = take((size_t)L.nT * kNB * kNB * rs);
  L.sync = take((size_t)chol_sync_ints(L.nT) * 4);
  L.gains = take(K * N * 8 * rs);
  L.gain_inv = take(N * 8 * rs);
  L.parts = take((size_t)kMaxParts * 8);
  L.srcp = take(F * Smax * 32);
  L.pen = take(K * 8 * N * 8);
  L.total = o;
  return L;
}

// ---- argument checks -----------------------------------------------------------------------

static int check_dims(const sc_dims* d, int32_t prec, Shape& s) {
  if (d == nullptr) return fail(SC_EINVAL, "dims is NULL");
  if (prec != SC_FP64 && prec != SC_MIXED) return fail(SC_EINVAL, "unknown precision %d", prec);
  if (d->N < 2 || d->N > 8000) return fail(SC_EINVAL, "N = %d outside [2, 8000]", d->N);
  if (d->T < 1 || d->F < 1 || d->K < 1) return fail(SC_EINVAL, "T, F, K must be >= 1 (T=%d F=%d K=%d)", d->T, d->F, d->K);
  if ((int64_t)d->T * d->F > 65535) return fail(SC_EINVAL, "T*F = %lld exceeds 65535", (long long)d->T * d->F);
  if (d->S_max < 0 || d->S_max > 65535) return fail(SC_EINVAL, "S_max = %d outside [0, 65535]", d->S_max);
  s.N = d->N;
  s.T = d->T;
  s.F = d->F;
  s.K = d->K;
  s.S_max = d->S_max;
  s.B = (int64_t)d->N * (d->N - 1) / 2;
  s.prec = prec;
  return SC_OK;
}

struct Ctx {
  Shape s;
  Workspace L;
  char* base;
  cudaStream_t st;
  int splits;  // coherency splits for the current device (<= L.splits)
  template <class T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(base + off);
  }
  uint32_t* status() const { return at<uint32_t>(L.status); }
  LMState* lm() const { return at<LMState>(L.lm); }
};

static int open_ctx(Ctx& c, const sc_dims* d, int32_t prec, void* ws, size_t ws_bytes, void* stream) {
  int r = check_dims(d, prec, c.s);
  if (r) return r;
  if (ws == nullptr) return fail(SC_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(SC_EINVAL, "workspace not 256-byte aligned");
  c.L = plan_workspace(c.s, true);
  if (ws_bytes < c.L.total)
    return fail(SC_ENOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, c.L.total);
  c.base = static_cast<char*>(ws);
  c.st = static_cast<cudaStream_t>(stream);
  c.splits = std::min(c.L.splits, coherency_splits(c.s, device_sms()));
  SC_CUDA(cudaMemsetAsync(c.status(), 0, 256, c.st));
  return SC_OK;
}

static int check_sky(const Shape& s, const sc_sky* sky) {
  if (sky == nullptr || sky->offsets == nullptr) return fail(SC_EINVAL, "sky or sky->offsets is NULL");
  if (sky->offsets[0] != 0) return fail(SC_EINVAL, "sky->offsets[0] must be 0");
  for (int k = 0; k < s.K; ++k) {
    int n = sky->offsets[k + 1] - sky->offsets[k];
    if (n < 0) return fail(SC_EINVAL, "sky->offsets decreases at cluster %d", k);
    if (n > s.S_max) return fail(SC_EINVAL, "cluster %d has %d sources > S_max = %d", k, n, s.S_max);
  }
  if (sky->offsets[s.K] > 0 && (!sky->l || !sky->m || !sky->flux || !sky->alpha))
    return fail(SC_EINVAL, "sky source arrays must not be NULL");
  if (!(sky->f0 > 0)) return fail(SC_EINVAL, "sky->f0 must be > 0");
  return SC_OK;
}

static int check_sky_full(const Shape& s, const sc_sky_full* sky) {
  if (sky == nullptr || sky->offsets == nullptr) return fail(SC_EINVAL, "sky or sky->offsets is NULL");
  if (sky->offsets[0] != 0) return fail(SC_EINVAL, "sky->offsets[0] must be 0");
  for (int k = 0; k < s.K; ++k) {
    int n = sky->offsets[k + 1] - sky->offsets[k];
    if (n < 0) return fail(SC_EINVAL, "sky->offsets decreases at cluster %d", k);
    if (n > s.S_max) return fail(SC_EINVAL, "cluster %d has %d sources > S_max = %d", k, n, s.S_max);
  }
  if (sky->offsets[s.K] > 0 && (!sky->l || !sky->m || !sky->I || !sky->Q || !sky->U || !sky->V ||
                                !sky->alpha || !sky->maj || !sky->mnr || !sky->pa))
    return fail(SC_EINVAL, "sky source arrays must not be NULL");
  if (!(sky->f0 > 0)) return fail(SC_EINVAL, "sky->f0 must be > 0");
  if ((int64_t)s.F * std::max(s.S_max, 1) > (int64_t(1) << 30))
    return fail(SC_EINVAL, "F * S_max = %lld exceeds 2^30", (long long)s.F * s.S_max);
  return SC_OK;
}

static int check_lm(const sc_lm_opts* o) {
  if (o == nullptr) return fail(SC_EINVAL, "LM options are NULL");
  if (o->n_lm < 0 || o->refine_sweeps < 0 || o->refine_sweeps > 16)
    return fail(SC_EINVAL, "n_lm must be >= 0 and refine_sweeps in [0, 16]");
  if (!(o->tau > 0)) return fail(SC_EINVAL, "tau must be > 0");
  if (!(o->eps_grad >= 0)) return fail(SC_EINVAL, "eps_grad must be >= 0");
  if (o->max_ctas < 0) return fail(SC_EINVAL, "max_ctas must be >= 0");
  if (o->chol_kernel != SC_CHOL_SIMT && o->chol_kernel != SC_CHOL_TENSOR)
    return fail(SC_EINVAL, "chol_kernel = %d is neither SC_CHOL_SIMT nor SC_CHOL_TENSOR", o->chol_kernel);
  return SC_OK;
}

// ---- pieces of the path ----------------------------------------------------------------------

// Coherencies of every cluster into C_out [K][T][B][F]; w_out [K][B] if not NULL.
template <typename R>
static int predict_all(const Ctx& c, const double* uvw, const double* freqs, const sc_sky* sky,
                       R* C_out, R* w_out) {
  const Shape& s = c.s;
  size_t per = (size_t)s.T * s.B * s.F * 2;
  for (int k = 0; k < s.K; ++k) {
    int a = sky->offsets[k], S = sky->offsets[k + 1] - a;
    R* Ck = C_out + per * k;
    if (s.prec == SC_MIXED) {
      float2* E = c.at<float2>(c.L.E);
      float* Sf = c.at<float>(c.L.Sf);
      float* wpart = c.at<float>(c.L.wpart);
      SC_LAUNCH(PK_PHASORS, launch_station_phasors(s, uvw, freqs, sky->l + a, sky->m + a, sky->flux + a,
                                     sky->alpha + a, sky->f0, S, E, Sf, c.st));
      SC_LAUNCH(PK_COHERENCY, launch_coherency_f32(s, S, E, Sf, reinterpret_cast<float2*>(Ck), wpart, c.splits, c.st));
      if (w_out)
        SC_LAUNCH(PK_OTHER, launch_sum_parts(wpart, c.splits, s.B, reinterpret_cast<float*>(w_out) + (size_t)s.B * k,
                                 c.st));
    } else {
      if (S > 0) {
        SC_LAUNCH(PK_COHERENCY, launch_predict_f64(s, uvw, freqs, sky->l + a, sky->m + a, sky->flux + a, sky->alpha + a,
                                   sky->f0, S, reinterpret_cast<double2*>(Ck), c.st));
      } else {
        SC_CUDA(cudaMemsetAsync(Ck, 0, per * sizeof(R), c.st));
      }
      if (w_out)
        SC_LAUNCH(PK_OTHER, launch_w_from_C<R>(s, Ck, w_out + (size_t)s.B * k, c.st));
    }
  }
  return SC_OK;
}

// Full 2x2 coherencies of every cluster of a polarised sky into C_out [K][T][B][F][2][2].
template <typename R>
static int predict_full_all(const Ctx& c, const double* uvw, const double* freqs, const sc_sky_full* sky,
                            R* C_out) {
  const Shape& s = c.s;
  const size_t per = (size_t)s.T * s.B * s.F * 8;
  for (int k = 0; k < s.K; ++k) {
    const int a = sky->offsets[k], S = sky->offsets[k + 1] - a;
    const SkyFull kf{sky->l + a, sky->m + a, sky->I + a, sky->Q + a, sky->U + a, sky->V + a,
                     sky->alpha + a, sky->maj + a, sky->mnr + a, sky->pa + a, sky->f0};
    R* Ck = C_out + per * k;
    if (s.prec == SC_MIXED) {
      float2* E = c.at<float2>(c.L.E);
      float* Sf = c.at<float>(c.L.Sf);
      float4* stp = c.at<float4>(c.L.srcp);
      float4* gqp = stp + (size_t)s.F * std::max(s.S_max, 1);
      SC_LAUNCH(PK_PHASORS, launch_station_phasors(s, uvw, freqs, kf.l, kf.m, kf.I, kf.alpha, kf.f0, S, E, Sf,
                                                   c.st));
      SC_LAUNCH(PK_OTHER, launch_source_params(s, S, freqs, kf, stp, gqp, c.st));
      SC_LAUNCH(PK_COHERENCY,
                launch_coherency_full_f32(s, S, uvw, E, stp, gqp, reinterpret_cast<float*>(Ck), c.st));
    } else {
      SC_LAUNCH(PK_COHERENCY, launch_predict_full_f64(s, S, uvw, freqs, kf, reinterpret_cast<double*>(Ck), c.st));
    }
  }
  return SC_OK;
}

// Levenberg-Marquardt on one cluster.  Data: X = Xin (running = false) or
// X = Xin + c J_old J_old^H with J_old the Jones at entry (running = true,
// Xin being the residual of all clusters).  J_io [8N] in/out.  pen [8N],
// if not NULL, adds pen_w |theta - pen|^2 to the cost.
template <typename R>
static int lm_solve(const Ctx& c, const R* Xin, bool running, const R* C, const R* w, double* J_io,
                    const sc_lm_opts& o, double* cost_out, int32_t* iters_out, const double* pen = nullptr,
                    double pen_w = 0.0) {
  const Shape& s = c.s;
  const Workspace& L = c.L;
  size_t n8 = (size_t)8 * s.N * sizeof(double);
  const bool mixed = s.prec == SC_MIXED;
  LMBufs b{};
  b.J_cur = c.at<double>(L.J_cur);
  b.J_trial = c.at<double>(L.J_trial);
  b.g_cur = c.at<double>(L.g_cur);
  b.g_trial = c.at<double>(L.g_trial);
  b.H_cur = c.at<double>(L.H_cur);
  b.H_trial = c.at<double>(L.H_trial);
  b.cp_cur = c.at<double>(L.cpart_cur);
  b.cp_trial = c.at<double>(L.cpart_trial);
  b.gm_cur = c.at<double>(L.gm_cur);
  b.gm_trial = c.at<double>(L.gm_trial);
  b.pred_part = c.at<double>(L.pred_part);
  b.Jf_cur = mixed ? c.at<float>(L.Jf_cur) : nullptr;
  b.Jf_trial = mixed ? c.at<float>(L.Jf_trial) : nullptr;
  // the Jones in the matrix's type for the assembly of J^T J
  const R* Jr = nullptr;
  if constexpr (sizeof(R) == 4) Jr = b.Jf_cur;
  else Jr = b.J_cur;
  double* J_old = c.at<double>(L.J_old);
  double* x = c.at<double>(L.x);
  double* rvec = c.at<double>(L.rvec);
  double* stat = c.at<double>(L.lstat);
  double* part = c.at<double>(L.part);
  R* A = c.at<R>(L.A);
  R* Linv = c.at<R>(L.Linv);
  uint64_t* bw = c.at<uint64_t>(L.bvec);
  int* sync = c.at<int>(L.sync);
  LMState* lm = c.lm();

  SC_CUDA(cudaMemcpyAsync(J_old, J_io, n8, cudaMemcpyDeviceToDevice, c.st));
  SC_CUDA(cudaMemcpyAsync(b.J_cur, J_io, n8, cudaMemcpyDeviceToDevice, c.st));
  SC_CUDA(cudaMemsetAsync(x, 0, (size_t)L.Ppad * sizeof(double), c.st));
  SC_CUDA(cudaMemsetAsync(rvec, 0, (size_t)L.Ppad * sizeof(double), c.st));
  SC_CUDA(cudaMemsetAsync(bw, 0, (size_t)L.Ppad * 2 * sizeof(R), c.st));  // no stale tag can match
  int nst = 0;  // timeslot chunks of the statistics
  SC_LAUNCH(PK_STATS, launch_lm_stats<R>(s, Xin, C, running ? J_old : nullptr, stat, &nst, c.st));
  SC_LAUNCH(PK_REDUCE, launch_lm_eval<R>(s, true, stat, nst, b.J_cur, part, nullptr, c.st));
  SC_LAUNCH(PK_REDUCE, launch_station_sum(s, part, b.J_cur, b.g_cur, b.H_cur, b.cp_cur, b.gm_cur, nullptr, pen, pen_w,
                                          c.st));
  SC_LAUNCH(PK_LM, launch_lm_init(lm, &o, s.N, b, b.J_cur, c.st));
  for (int it = 0; it < o.n_lm; ++it) {
    SC_LAUNCH(PK_ASSEMBLE, launch_assemble<R>(s, L.Ppad, L.Ppad, w, Jr, b.H_cur, lm, A, true, false, c.st));
    SC_LAUNCH(PK_CHOL, launch_chol<R>(A, L.Ppad, L.nT, Linv, sync, c.status(), lm, o.max_ctas, o.chol_kernel, c.st));
    SC_LAUNCH(PK_SOLVE, launch_chol_solve<R>(A, L.Ppad, L.nT, Linv, sync, b.g_cur, bw, x, 0, c.status(), lm, c.st));
    if (mixed) {
      for (int sw = 0; sw < o.refine_sweeps; ++sw) {
        SC_LAUNCH(PK_REFINE, launch_refine_residual<R>(s, w, b.J_cur, b.H_cur, b.g_cur, x, lm, c.at<double>(L.ry),
                                                       rvec, c.st));
        SC_LAUNCH(PK_SOLVE, launch_chol_solve<R>(A, L.Ppad, L.nT, Linv, sync, rvec, bw, x, 1, c.status(), lm, c.st));
      }
    }
    SC_LAUNCH(PK_LM, launch_lm_trial(lm, s.N, x, b, c.st));
    SC_LAUNCH(PK_REDUCE, launch_lm_eval<R>(s, true, stat, nst, b.J_trial, part, lm, c.st));
    SC_LAUNCH(PK_REDUCE, launch_station_sum(s, part, b.J_trial, b.g_trial, b.H_trial, b.cp_trial, b.gm_trial, lm, pen,
                                            pen_w, c.st));
    SC_LAUNCH(PK_LM, launch_lm_decide(lm, s.N, b, c.st));
  }
  SC_LAUNCH(PK_LM, launch_lm_finish(lm, b.J_cur, s.N, J_io, cost_out, iters_out, c.st));
  return SC_OK;
}

// pen [K][8N], if not NULL, adds pen_w |J_k - pen_k|^2 to cluster k's LM cost.
template <typename R>
static int sage(const Ctx& c, const double* uvw, const double* freqs, const sc_sky* sky, const R* V,
                double* jones, const sc_sage_opts& o, double* costs, const double* pen = nullptr,
                double pen_w = 0.0) {
  const Shape& s = c.s;
  const Workspace& L = c.L;
  R* C = c.at<R>(L.C);
  R* w = c.at<R>(L.w);
  R* Rres = c.at<R>(L.Rres);
  size_t perC = (size_t)s.T * s.B * s.F * 2;
  size_t perV = (size_t)s.T * s.B * s.F * 8;
  int r = predict_all<R>(c, uvw, freqs, sky, C, w);
  if (r) return r;
  // running residual R = V - sum_k model_k
  SC_CUDA(cudaMemcpyAsync(Rres, V, perV * sizeof(R), cudaMemcpyDeviceToDevice, c.st));
  for (int k = 0; k < s.K; ++k)
    SC_LAUNCH(PK_PASS, launch_pass<R>(s, P_SUB | P_WRITE_R, Rres, C + perC * k, nullptr, jones + (size_t)8 * s.N * k, Rres,
                           nullptr, nullptr, L.nchunk, L.tchunk, nullptr, c.st));
  for (int em = 0; em < o.n_em; ++em) {
    for (int k = 0; k < s.K; ++k) {
      double* Jk = jones + (size_t)8 * s.N * k;
      const R* Ck = C + perC * k;
      r = lm_solve<R>(c, Rres, true, Ck, w + (size_t)s.B * k, Jk, o.lm, costs ? costs + k : nullptr, nullptr,
                      pen ? pen + (size_t)8 * s.N * k : nullptr, pen_w);
      if (r) return r;
      // R += c (J_old J_old^H - J_new J_new^H)
      SC_LAUNCH(PK_PASS, launch_pass<R>(s, P_OLD | P_SUB | P_WRITE_R, Rres, Ck, c.at<double>(L.J_old), Jk, Rres, nullptr,
                             nullptr, L.nchunk, L.tchunk, nullptr, c.st));
    }
  }
  return SC_OK;
}

template <typename R>
static int residual_impl(const Ctx& c, const void* X, const void* C, const double* jones, void* Rout,
                         double* cost) {
  const Workspace& L = c.L;
  int flags = P_SUB | (Rout ? P_WRITE_R : 0) | (cost ? P_STATS : 0);
  if (!(flags & (P_WRITE_R | P_STATS))) return SC_OK;
  if (flags == (P_SUB | P_STATS)) {
    SC_LAUNCH(PK_PASS, launch_pass<R>(c.s, P_SUB | P_STATS, static_cast<const R*>(X), static_cast<const R*>(C), nullptr, jones,
                           nullptr, c.at<R>(L.stat_cost), c.at<R>(L.stat_rho), L.nchunk, L.tchunk, nullptr, c.st));
  } else {
    SC_LAUNCH(PK_PASS, launch_pass<R>(c.s, flags, static_cast<const R*>(X), static_cast<const R*>(C), nullptr, jones,
                           static_cast<R*>(Rout), c.at<R>(L.stat_cost), c.at<R>(L.stat_rho), L.nchunk, L.tchunk,
                           nullptr, c.st));
  }
  if (cost) SC_LAUNCH(PK_OTHER, launch_sum_reals<R>(c.at<R>(L.stat_cost), (int64_t)L.nchunk * c.s.B, cost, c.st));
  return SC_OK;
}

template <typename R>
static int residual_all_impl(const Ctx& c, const void* V, const void* C, const double* jones, int corr,
                             void* Rout, double* cost) {
  const Workspace& L = c.L;
  R* Jr = c.at<R>(L.gains);
  R* Jinv = c.at<R>(L.gain_inv);
  double* part = cost ? c.at<double>(L.parts) : nullptr;
  int n_parts = 0;
  SC_LAUNCH(PK_OTHER, launch_gain_prep<R>(c.s, jones, corr, Jr, Jinv, c.status(), c.st));
  SC_LAUNCH(PK_PASS, launch_residual_all<R>(c.s, static_cast<const R*>(V), static_cast<const R*>(C), Jr,
                                            corr >= 0 ? Jinv : nullptr, static_cast<R*>(Rout), part,
                                            kMaxParts, &n_parts, c.st));
  if (cost) SC_LAUNCH(PK_OTHER, launch_sum_cost(part, n_parts, cost, c.st));
  return SC_OK;
}

template <typename R>
static int normal_eqs_impl(const Ctx& c, const void* Rv, const void* C, const double* jones, void* JhJ,
                           double* Jhr) {
  const Workspace& L = c.L;
  const Shape& s = c.s;
  R* w = c.at<R>(L.w);
  SC_LAUNCH(PK_OTHER, launch_w_from_C<R>(s, static_cast<const R*>(C), w, c.st));
  int nst = 0;
  double* stat = c.at<double>(L.lstat);
  double* part = c.at<double>(L.part);
  SC_LAUNCH(PK_STATS, launch_lm_stats<R>(s, static_cast<const R*>(Rv), static_cast<const R*>(C), nullptr, stat, &nst,
                                         c.st));
  SC_LAUNCH(PK_REDUCE, launch_lm_eval<R>(s, false, stat, nst, jones, part, nullptr, c.st));
  SC_LAUNCH(PK_REDUCE, launch_station_sum(s, part, jones, Jhr, c.at<double>(L.H_cur), c.at<double>(L.cpart_cur),
                                          c.at<double>(L.gm_cur), nullptr, nullptr, 0.0, c.st));
  int P = 8 * s.N;
  const R* Jr = nullptr;
  if constexpr (sizeof(R) == 4) {
    SC_LAUNCH(PK_OTHER, launch_round_jones(jones, c.at<float>(L.Jf_cur), 8 * s.N, c.st));
    Jr = c.at<float>(L.Jf_cur);
  } else {
    Jr = jones;
  }
  SC_LAUNCH(PK_ASSEMBLE, launch_assemble<R>(s, P, P, w, Jr, c.at<double>(L.H_cur), nullptr, static_cast<R*>(JhJ), false,
                                            true, c.st));
  return SC_OK;
}

// Internal streams and events for the concurrent bands of the consensus
// call, created once per device and kept for the life of the process.
constexpr int kConsensusStreams = 16;
static int consensus_streams(int m, cudaStream_t* st, cudaEvent_t* fork, cudaEvent_t* joins) {
  constexpr int kDevs = 64;
  struct Pool {
    cudaStream_t s[kConsensusStreams];
    cudaEvent_t fork, join[kConsensusStreams];
    bool made;
  };
  static Pool pools[kDevs];
  static std::mutex mu;
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kDevs) return fail(SC_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(mu);
  Pool& p = pools[dev];
  if (!p.made) {
    for (int k = 0; k < kConsensusStreams; ++k) {
      SC_CUDA(cudaStreamCreateWithFlags(&p.s[k], cudaStreamNonBlocking));
      SC_CUDA(cudaEventCreateWithFlags(&p.join[k], cudaEventDisableTiming));
    }
    SC_CUDA(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
    p.made = true;
  }
  for (int k = 0; k < m; ++k) st[k] = p.s[k], joins[k] = p.join[k];
  *fork = p.fork;
  return SC_OK;
}

// ---- lock-step batch -------------------------------------------------------------------------

// One job's block of a lock-step batch workspace: the buffers of a cluster
// solve (the fields of a job workspace that the LM loop uses, the cluster's
// w, statistics room for T_max timeslots).  Blocks follow each other at the
// stride L.total, so that one launch moves every pointer by job * stride.
static Workspace plan_lm_block(const Shape& s, int T_max) {
  Workspace L{};
  const size_t rs = s.prec == SC_MIXED ? 4 : 8;
  const size_t N = s.N, B = (size_t)s.B;
  L.Ppad = (int)((8 * N + kNB - 1) / kNB * kNB);
  L.nT = L.Ppad / kNB;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    size_t at = o;
    o = align256(o + std::max<size_t>(bytes, 1));
    return at;
  };
  L.status = take(256);
  L.lm = take(sizeof(LMState));
  L.w = take(B * rs);
  L.lstat = take(lm_stats_doubles(T_max, s.B) * 8);
  L.part = take(lm_part_doubles(s.N) * 8);
  L.J_old = take(8 * N * 8);
  L.J_cur = take(8 * N * 8);
  L.J_trial = take(8 * N * 8);
  L.g_cur = take(8 * N * 8);
  L.g_trial = take(8 * N * 8);
  L.H_cur = take(4 * N * 8);
  L.H_trial = take(4 * N * 8);
  L.cpart_cur = take(N * 8);
  L.cpart_trial = take(N * 8);
  L.gm_cur = take(N * 8);
  L.gm_trial = take(N * 8);
  L.pred_part = take((8 * N / 256 + 1) * 8);
  L.Jf_cur = take(8 * N * 4);
  L.Jf_trial = take(8 * N * 4);
  L.x = take((size_t)L.Ppad * 8);
  L.rvec = take((size_t)L.Ppad * 8);
  L.ry = take((size_t)L.Ppad * 8);
  L.bvec = take((size_t)L.Ppad * 2 * rs);
  L.A = take((size_t)L.Ppad * L.Ppad * rs);
  L.Linv = take((size_t)L.nT * kNB * kNB * rs);
  L.sync = take((size_t)chol_sync_ints(L.nT) * 4);
  L.total = o;
  return L;
}

// A lock-step batch workspace: G job blocks, then the combined task order
// of the factorisation (G x tasks per job, uint32) when one can be formed.
struct BatchedLayout {
  Workspace block;
  size_t order;  // offset of the order table; 0 if none
  size_t total;
};
static BatchedLayout plan_batched(const Shape& s0, int T_max, int G) {
  BatchedLayout b;
  b.block = plan_lm_block(s0, T_max);
  b.total = b.block.total * (size_t)G;
  b.order = 0;
  if (batch_order_ok(b.block.nT, G)) {
    b.order = b.total;
    b.total += align256((size_t)chol_ntasks(b.block.nT) * G * sizeof(uint32_t));
  }
  return b;
}

// SAGE on every job of a lock-step batch (equal N and K), all on c.st.
// c: the batch workspace (c.L a block layout, c.s the shape of job 0);
// jc: the jobs' own workspaces (coherencies, w, running residual).  Per
// cluster, each job's statistics pass runs on its own data; then each LM
// stage is one launch over all jobs, the factorisations one persistent
// kernel; then each job's Jones and residual are updated.  Every job's
// arithmetic is that of sage() alone.
template <typename R>
static int sage_batched(const Ctx& c, const std::vector<Ctx>& jc, const sc_job* jobs, const sc_sage_opts& o,
                        const uint32_t* order) {
  const int G = (int)jc.size();
  const Shape& s = c.s;
  const Workspace& L = c.L;
  const size_t js = L.total;
  const Batch bt{G, js};
  const bool mixed = s.prec == SC_MIXED;
  const size_t n8 = (size_t)8 * s.N * sizeof(double);
  // job 0's buffers; the launches reach the others through the stride
  LMBufs b{};
  b.J_cur = c.at<double>(L.J_cur);
  b.J_trial = c.at<double>(L.J_trial);
  b.g_cur = c.at<double>(L.g_cur);
  b.g_trial = c.at<double>(L.g_trial);
  b.H_cur = c.at<double>(L.H_cur);
  b.H_trial = c.at<double>(L.H_trial);
  b.cp_cur = c.at<double>(L.cpart_cur);
  b.cp_trial = c.at<double>(L.cpart_trial);
  b.gm_cur = c.at<double>(L.gm_cur);
  b.gm_trial = c.at<double>(L.gm_trial);
  b.pred_part = c.at<double>(L.pred_part);
  b.Jf_cur = mixed ? c.at<float>(L.Jf_cur) : nullptr;
  b.Jf_trial = mixed ? c.at<float>(L.Jf_trial) : nullptr;
  const R* Jr = nullptr;
  if constexpr (sizeof(R) == 4) Jr = b.Jf_cur;
  else Jr = b.J_cur;
  double* x = c.at<double>(L.x);
  double* rvec = c.at<double>(L.rvec);
  double* stat = c.at<double>(L.lstat);
  double* part = c.at<double>(L.part);
  R* w = c.at<R>(L.w);
  R* A = c.at<R>(L.A);
  R* Linv = c.at<R>(L.Linv);
  uint64_t* bw = c.at<uint64_t>(L.bvec);
  int* sync = c.at<int>(L.sync);
  LMState* lm = c.lm();
  const int* nchunk_dev = &lm->nchunk;
  auto blk = [&](int g) { return c.base + (size_t)g * js; };

  // every job: coherencies and w, running residual R = V - sum_k model_k
  SC_CUDA(cudaMemset2DAsync(c.base + L.status, js, 0, 256, G, c.st));
  for (int g = 0; g < G; ++g) {
    const Ctx& j = jc[g];
    const size_t perC = (size_t)j.s.T * j.s.B * j.s.F * 2, perV = (size_t)j.s.T * j.s.B * j.s.F * 8;
    R* C = j.at<R>(j.L.C);
    R* Rres = j.at<R>(j.L.Rres);
    int r = predict_all<R>(j, jobs[g].uvw, jobs[g].freqs, &jobs[g].sky, C, j.at<R>(j.L.w));
    if (r) return r;
    SC_CUDA(cudaMemcpyAsync(Rres, jobs[g].V, perV * sizeof(R), cudaMemcpyDeviceToDevice, c.st));
    for (int k = 0; k < s.K; ++k)
      SC_LAUNCH(PK_PASS, launch_pass<R>(j.s, P_SUB | P_WRITE_R, Rres, C + perC * k, nullptr,
                                        jobs[g].jones + (size_t)8 * s.N * k, Rres, nullptr, nullptr, j.L.nchunk,
                                        j.L.tchunk, nullptr, c.st));
  }
  for (int em = 0; em < o.n_em; ++em) {
    for (int k = 0; k < s.K; ++k) {
      // per job: the cluster's Jones, w and statistics into its block
      for (int g = 0; g < G; ++g) {
        const Ctx& j = jc[g];
        const size_t perC = (size_t)j.s.T * j.s.B * j.s.F * 2;
        char* bg = blk(g);
        double* Jk = jobs[g].jones + (size_t)8 * s.N * k;
        double* J_old = reinterpret_cast<double*>(bg + L.J_old);
        SC_CUDA(cudaMemcpyAsync(J_old, Jk, n8, cudaMemcpyDeviceToDevice, c.st));
        SC_CUDA(cudaMemcpyAsync(bg + L.J_cur, Jk, n8, cudaMemcpyDeviceToDevice, c.st));
        SC_CUDA(cudaMemcpyAsync(bg + L.w, j.at<R>(j.L.w) + (size_t)s.B * k, (size_t)s.B * sizeof(R),
                                cudaMemcpyDeviceToDevice, c.st));
        int nst = 0;
        SC_LAUNCH(PK_STATS, launch_lm_stats<R>(j.s, j.at<R>(j.L.Rres), j.at<R>(j.L.C) + perC * k, J_old,
                                               reinterpret_cast<double*>(bg + L.lstat), &nst, c.st,
                                               reinterpret_cast<int*>(bg + L.lm + offsetof(LMState, nchunk))));
      }
      SC_CUDA(cudaMemset2DAsync(x, js, 0, (size_t)L.Ppad * sizeof(double), G, c.st));
      SC_CUDA(cudaMemset2DAsync(rvec, js, 0, (size_t)L.Ppad * sizeof(double), G, c.st));
      SC_CUDA(cudaMemset2DAsync(bw, js, 0, (size_t)L.Ppad * 2 * sizeof(R), G, c.st));  // no stale tag can match
      // the LM loop, one launch per stage for every job
      SC_LAUNCH(PK_REDUCE, launch_lm_eval<R>(s, true, stat, 0, b.J_cur, part, nullptr, c.st, bt, nchunk_dev));
      SC_LAUNCH(PK_REDUCE, launch_station_sum(s, part, b.J_cur, b.g_cur, b.H_cur, b.cp_cur, b.gm_cur, nullptr,
                                              nullptr, 0.0, c.st, bt));
      SC_LAUNCH(PK_LM, launch_lm_init(lm, &o.lm, s.N, b, b.J_cur, c.st, bt));
      for (int it = 0; it < o.lm.n_lm; ++it) {
        SC_LAUNCH(PK_ASSEMBLE, launch_assemble<R>(s, L.Ppad, L.Ppad, w, Jr, b.H_cur, lm, A, true, false, c.st, bt));
        SC_LAUNCH(PK_CHOL, launch_chol_batch<R>(A, L.Ppad, L.nT, Linv, sync, c.status(), lm, o.lm.max_ctas, bt,
                                                order, c.st));
        SC_LAUNCH(PK_SOLVE, launch_chol_solve<R>(A, L.Ppad, L.nT, Linv, sync, b.g_cur, bw, x, 0, c.status(), lm,
                                                 c.st, bt));
        if (mixed) {
          for (int sw = 0; sw < o.lm.refine_sweeps; ++sw) {
            SC_LAUNCH(PK_REFINE, launch_refine_residual<R>(s, w, b.J_cur, b.H_cur, b.g_cur, x, lm,
                                                           c.at<double>(L.ry), rvec, c.st, bt));
            SC_LAUNCH(PK_SOLVE, launch_chol_solve<R>(A, L.Ppad, L.nT, Linv, sync, rvec, bw, x, 1, c.status(), lm,
                                                     c.st, bt));
          }
        }
        SC_LAUNCH(PK_LM, launch_lm_trial(lm, s.N, x, b, c.st, bt));
        SC_LAUNCH(PK_REDUCE, launch_lm_eval<R>(s, true, stat, 0, b.J_trial, part, lm, c.st, bt, nchunk_dev));
        SC_LAUNCH(PK_REDUCE, launch_station_sum(s, part, b.J_trial, b.g_trial, b.H_trial, b.cp_trial, b.gm_trial,
                                                lm, nullptr, 0.0, c.st, bt));
        SC_LAUNCH(PK_LM, launch_lm_decide(lm, s.N, b, c.st, bt));
      }
      // per job: the new Jones and the residual R += c (J_old J_old^H - J_new J_new^H)
      for (int g = 0; g < G; ++g) {
        const Ctx& j = jc[g];
        const size_t perC = (size_t)j.s.T * j.s.B * j.s.F * 2;
        char* bg = blk(g);
        double* Jk = jobs[g].jones + (size_t)8 * s.N * k;
        SC_LAUNCH(PK_LM, launch_lm_finish(reinterpret_cast<LMState*>(bg + L.lm),
                                          reinterpret_cast<double*>(bg + L.J_cur), s.N, Jk,
                                          jobs[g].costs ? jobs[g].costs + k : nullptr, nullptr, c.st));
        R* Rres = j.at<R>(j.L.Rres);
        SC_LAUNCH(PK_PASS, launch_pass<R>(j.s, P_OLD | P_SUB | P_WRITE_R, Rres, j.at<R>(j.L.C) + perC * k,
                                          reinterpret_cast<double*>(bg + L.J_old), Jk, Rres, nullptr, nullptr,
                                          j.L.nchunk, j.L.tchunk, nullptr, c.st));
      }
    }
  }
  // each job's status word gathers its block's
  for (int g = 0; g < G; ++g)
    SC_LAUNCH(PK_OTHER, launch_or_status(reinterpret_cast<const uint32_t*>(blk(g) + L.status), jc[g].status(),
                                         c.st));
  return SC_OK;
}

}  // namespace sc

using namespace sc;

// ---- exported entry points ------------------------------------------------------------------

extern "C" {

SC_API int32_t sc_version(void) { return (1 << 16) | 0; }

SC_API int32_t sc_last_error(char* buf, size_t len) {
  if (buf && len) {
    strncpy(buf, g_msg, len - 1);
    buf[len - 1] = 0;
  }
  return g_err;
}

SC_API int32_t sc_workspace_size(const sc_dims* d, int32_t prec, size_t* bytes) {
  Shape s;
  int r = check_dims(d, prec, s);
  if (r) return r;
  if (!bytes) return fail(SC_EINVAL, "bytes is NULL");
  *bytes = plan_workspace(s, true).total;
  return ok();
}

SC_API int32_t sc_device_status(const void* ws, size_t ws_bytes, uint32_t* status) {
  if (!ws || !status || ws_bytes < 256) return fail(SC_EINVAL, "bad workspace or status pointer");
  // the status word is at offset 0 of every workspace layout
  SC_CUDA(cudaMemcpy(status, ws, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return ok();
}

SC_API uint64_t sc_launch_count(void) { return launch_count(); }

SC_API int32_t sc_profile_begin(void) {
  prof_begin();
  return ok();
}

SC_API int32_t sc_profile_end(void) {
  if (prof_end() != 0) return fail(SC_ECUDA, "profiling events could not be read");
  return ok();
}

SC_API int32_t sc_profile_read(int32_t kind, int64_t* launches, double* total_ms) {
  if (kind < 0 || kind >= PK_COUNT || !launches || !total_ms) return fail(SC_EINVAL, "bad profile query");
  long n = 0;
  double ms = 0;
  prof_read(kind, &n, &ms);
  *launches = n;
  *total_ms = ms;
  return ok();
}

SC_API int32_t sc_chol_schedule(int32_t nT, int32_t which, int32_t* out, int32_t cap) {
  if (nT < 1 || nT > 1024 || (which != 0 && which != 1)) return fail(SC_EINVAL, "bad nT or list");
  int n = which == 0 ? chol_ntasks(nT) : 2 * nT;
  if (out) {
    if (cap < n) return fail(SC_EINVAL, "capacity %d < %d tasks", cap, n);
    for (int t = 0; t < n; ++t) {
      int4 v = which == 0 ? chol_task(nT, t) : solve_task(nT, t);
      out[4 * t] = v.x;
      out[4 * t + 1] = v.y;
      out[4 * t + 2] = v.z;
      out[4 * t + 3] = v.w;
    }
  }
  ok();
  return n;
}

SC_API int32_t sc_predict_coherencies(const sc_dims* d, const double* uvw, const double* freqs,
                                      const sc_sky* sky, void* C, int32_t prec, void* ws,
                                      size_t ws_bytes, void* stream) {
  Ctx c;
  int r = open_ctx(c, d, prec, ws, ws_bytes, stream);
  if (r) return r;
  if ((r = check_sky(c.s, sky))) return r;
  if (!uvw || !freqs || !C) return fail(SC_EINVAL, "uvw, freqs and C must not be NULL");
  r = prec == SC_MIXED ? predict_all<float>(c, uvw, freqs, sky, static_cast<float*>(C), nullptr)
                       : predict_all<double>(c, uvw, freqs, sky, static_cast<double*>(C), nullptr);
  return r ? r : ok();
}

SC_API int32_t sc_predict_coherencies_full(const sc_dims* d, const double* uvw, const double* freqs,
                                           const sc_sky_full* sky, void* C, int32_t prec, void* ws,
                                           size_t ws_bytes, void* stream) {
  Ctx c;
  // argument checks first: they touch no device memory
  int r = check_dims(d, prec, c.s);
  if (r) return r;
  if ((r = check_sky_full(c.s, sky))) return r;
  if (!uvw || !freqs || !C) return fail(SC_EINVAL, "uvw, freqs and C must not be NULL");
  if ((r = open_ctx(c, d, prec, ws, ws_bytes, stream))) return r;
  r = prec == SC_MIXED ? predict_full_all<float>(c, uvw, freqs, sky, static_cast<float*>(C))
                       : predict_full_all<double>(c, uvw, freqs, sky, static_cast<double*>(C));
  return r ? r : ok();
}

SC_API int32_t sc_residual(const sc_dims* d, const void* X, const void* C, const double* jones, void* R,
                           double* cost, int32_t prec, void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int r = open_ctx(c, d, prec, ws, ws_bytes, stream);
  if (r) return r;
  if (!X || !C || !jones) return fail(SC_EINVAL, "X, C and jones must not be NULL");
  r = prec == SC_MIXED ? residual_impl<float>(c, X, C, jones, R, cost)
                       : residual_impl<double>(c, X, C, jones, R, cost);
  return r ? r : ok();
}

SC_API int32_t sc_residual_all(const sc_dims* d, const void* V, const void* C, const double* jones,
                               int32_t corr, void* R, double* cost, int32_t prec, void* ws,
                               size_t ws_bytes, void* stream) {
  Ctx c;
  // argument checks first: they touch no device memory
  int r = check_dims(d, prec, c.s);
  if (r) return r;
  if (!V || !C || !jones || !R) return fail(SC_EINVAL, "V, C, jones and R must not be NULL");
  if (corr < -1 || corr >= c.s.K) return fail(SC_EINVAL, "corr = %d outside [-1, K = %d)", corr, c.s.K);
  if ((r = open_ctx(c, d, prec, ws, ws_bytes, stream))) return r;
  r = prec == SC_MIXED ? residual_all_impl<float>(c, V, C, jones, corr, R, cost)
                       : residual_all_impl<double>(c, V, C, jones, corr, R, cost);
  return r ? r : ok();
}

SC_API int32_t sc_lm_normal_eqs(const sc_dims* d, const void* R, const void* C, const double* jones, void* JhJ,
                                double* Jhr, int32_t prec, void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int r = open_ctx(c, d, prec, ws, ws_bytes, stream);
  if (r) return r;
  if (!R || !C || !jones || !JhJ || !Jhr) return fail(SC_EINVAL, "R, C, jones, JhJ and Jhr must not be NULL");
  r = prec == SC_MIXED ? normal_eqs_impl<float>(c, R, C, jones, JhJ, Jhr)
                       : normal_eqs_impl<double>(c, R, C, jones, JhJ, Jhr);
  return r ? r : ok();
}

}  // extern "C"

namespace sc {

// Layout of the workspace of sc_cholesky_solve.
struct CholWs {
  size_t status, A, Linv, sync, bvec, bpad, xpad, total;
  int Ppad, nT;
};
static CholWs plan_chol_ws(int n, int prec) {
  CholWs L{};
  const size_t rs = prec == SC_MIXED ? 4 : 8;
  L.Ppad = (n + kNB - 1) / kNB * kNB;
  L.nT = L.Ppad / kNB;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + std::max<size_t>(bytes, 1));
    return at;
  };
  L.status = take(256);
  L.A = take((size_t)L.Ppad * L.Ppad * rs);
  L.Linv = take((size_t)L.nT * kNB * kNB * rs);
  L.sync = take((size_t)chol_sync_ints(L.nT) * 4);
  L.bvec = take((size_t)L.Ppad * 2 * rs);
  L.bpad = take((size_t)L.Ppad * 8);
  L.xpad = take((size_t)L.Ppad * 8);
  L.total = o;
  return L;
}

template <typename R>
static int cholesky_impl(int n, R* A, int lda, const double* b, double* x, int kernel, const CholWs& L, char* base,
                         cudaStream_t st) {
  R* Aw = reinterpret_cast<R*>(base + L.A);
  R* Linv = reinterpret_cast<R*>(base + L.Linv);
  uint32_t* status = reinterpret_cast<uint32_t*>(base + L.status);
  double* bpad = reinterpret_cast<double*>(base + L.bpad);
  double* xpad = reinterpret_cast<double*>(base + L.xpad);
  uint64_t* bw = reinterpret_cast<uint64_t*>(base + L.bvec);
  int* sync = reinterpret_cast<int*>(base + L.sync);
  SC_CUDA(cudaMemsetAsync(status, 0, 256, st));
  // padded copy: A in the leading n x n block, identity beyond it
  SC_CUDA(cudaMemsetAsync(Aw, 0, (size_t)L.Ppad * L.Ppad * sizeof(R), st));
  SC_CUDA(cudaMemcpy2DAsync(Aw, (size_t)L.Ppad * sizeof(R), A, (size_t)lda * sizeof(R), (size_t)n * sizeof(R), n,
                            cudaMemcpyDeviceToDevice, st));
  SC_CUDA(launch_pad_identity<R>(Aw, L.Ppad, n, st));
  SC_CUDA(cudaMemsetAsync(sync, 0, (size_t)chol_sync_ints(L.nT) * 4, st));
  prof_start(PK_CHOL, st);
  const cudaError_t ce = launch_chol<R>(Aw, L.Ppad, L.nT, Linv, sync, status, nullptr, 0, kernel, st);
  prof_stop(PK_CHOL, st);
  SC_CUDA(ce);
  if (b != nullptr && x != nullptr) {
    SC_CUDA(cudaMemsetAsync(bpad, 0, (size_t)L.Ppad * 8, st));
    SC_CUDA(cudaMemcpyAsync(bpad, b, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
    SC_CUDA(cudaMemsetAsync(bw, 0, (size_t)L.Ppad * 2 * sizeof(R), st));
    prof_start(PK_SOLVE, st);
    const cudaError_t se = launch_chol_solve<R>(Aw, L.Ppad, L.nT, Linv, sync, bpad, bw, xpad, 0, status, nullptr, st);
    prof_stop(PK_SOLVE, st);
    SC_CUDA(se);
    SC_CUDA(cudaMemcpyAsync(x, xpad, (size_t)n * 8, cudaMemcpyDeviceToDevice, st));
  }
  SC_CUDA(cudaMemcpy2DAsync(A, (size_t)lda * sizeof(R), Aw, (size_t)L.Ppad * sizeof(R), (size_t)n * sizeof(R), n,
                            cudaMemcpyDeviceToDevice, st));
  return SC_OK;
}

}  // namespace sc

extern "C" {

SC_API int32_t sc_cholesky_workspace_size(int32_t n, int32_t prec, size_t* bytes) {
  if (n < 1 || n > 65536) return fail(SC_EINVAL, "n = %d outside [1, 65536]", n);
  if (prec != SC_FP64 && prec != SC_MIXED) return fail(SC_EINVAL, "unknown precision %d", prec);
  if (!bytes) return fail(SC_EINVAL, "bytes is NULL");
  *bytes = plan_chol_ws(n, prec).total;
  return ok();
}

SC_API int32_t sc_cholesky_solve(int32_t n, void* A, int32_t lda, const double* b, double* x, int32_t prec,
                                 int32_t chol_kernel, void* ws, size_t ws_bytes, void* stream) {
  if (n < 1 || n > 65536) return fail(SC_EINVAL, "n = %d outside [1, 65536]", n);
  if (prec != SC_FP64 && prec != SC_MIXED) return fail(SC_EINVAL, "unknown precision %d", prec);
  if (chol_kernel != SC_CHOL_SIMT && chol_kernel != SC_CHOL_TENSOR)
    return fail(SC_EINVAL, "chol_kernel = %d is neither SC_CHOL_SIMT nor SC_CHOL_TENSOR", chol_kernel);
  if (A == nullptr || lda < n) return fail(SC_EINVAL, "A is NULL or lda = %d < n = %d", lda, n);
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255)) return fail(SC_EINVAL, "workspace NULL or not 256-byte aligned");
  const CholWs L = plan_chol_ws(n, prec);
  if (ws_bytes < L.total) return fail(SC_ENOMEM, "workspace of %zu bytes, %zu needed", ws_bytes, L.total);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  char* base = static_cast<char*>(ws);
  const int r = prec == SC_MIXED ? cholesky_impl<float>(n, static_cast<float*>(A), lda, b, x, chol_kernel, L, base, st)
                                 : cholesky_impl<double>(n, static_cast<double*>(A), lda, b, x, chol_kernel, L, base,
                                                         st);
  return r ? r : ok();
}

SC_API int32_t sc_solve_cluster(const sc_dims* d, const void* X, const void* C, double* jones,
                                const sc_lm_opts* opts, double* cost, int32_t* iters, int32_t prec, void* ws,
                                size_t ws_bytes, void* stream) {
  Ctx c;
  int r = open_ctx(c, d, prec, ws, ws_bytes, stream);
  if (r) return r;
  if ((r = check_lm(opts))) return r;
  if (!X || !C || !jones) return fail(SC_EINVAL, "X, C and jones must not be NULL");
  if (prec == SC_MIXED) {
    float* w = c.at<float>(c.L.w);
    SC_LAUNCH(PK_OTHER, launch_w_from_C<float>(c.s, static_cast<const float*>(C), w, c.st));
    r = lm_solve<float>(c, static_cast<const float*>(X), false, static_cast<const float*>(C), w, jones, *opts, cost,
                        iters);
  } else {
    double* w = c.at<double>(c.L.w);
    SC_LAUNCH(PK_OTHER, launch_w_from_C<double>(c.s, static_cast<const double*>(C), w, c.st));
    r = lm_solve<double>(c, static_cast<const double*>(X), false, static_cast<const double*>(C), w, jones, *opts,
                         cost, iters);
  }
  return r ? r : ok();
}

SC_API int32_t sc_calibrate_sage(const sc_dims* d, const double* uvw, const double* freqs, const sc_sky* sky,
                                 const void* V, double* jones, const sc_sage_opts* opts, double* costs,
                                 int32_t prec, void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  int r = open_ctx(c, d, prec, ws, ws_bytes, stream);
  if (r) return r;
  if ((r = check_sky(c.s, sky))) return r;
  if (!opts) return fail(SC_EINVAL, "options are NULL");
  if (opts->n_em < 0) return fail(SC_EINVAL, "n_em must be >= 0");
  if ((r = check_lm(&opts->lm))) return r;
  if (!uvw || !freqs || !V || !jones) return fail(SC_EINVAL, "uvw, freqs, V and jones must not be NULL");
  r = prec == SC_MIXED
          ? sage<float>(c, uvw, freqs, sky, static_cast<const float*>(V), jones, *opts, costs)
          : sage<double>(c, uvw, freqs, sky, static_cast<const double*>(V), jones, *opts, costs);
  return r ? r : ok();
}

SC_API int32_t sc_calibrate_chunks(const sc_dims* d, int32_t n_chunks, const double* uvw,
                                   const double* freqs, const sc_sky* sky, const void* V,
                                   double* jones, double* jones_out, const sc_sage_opts* opts,
                                   double* costs, int32_t prec, void* ws, size_t ws_bytes,
                                   void* stream) {
  Ctx c;
  // argument checks first: they touch no device memory
  int r = check_dims(d, prec, c.s);
  if (r) return r;
  if (n_chunks < 1 || (int64_t)n_chunks * d->T > 65535)
    return fail(SC_EINVAL, "n_chunks = %d: need 1 <= n_chunks and n_chunks * T <= 65535", n_chunks);
  if ((r = check_sky(c.s, sky))) return r;
  if (!opts) return fail(SC_EINVAL, "options are NULL");
  if (opts->n_em < 0) return fail(SC_EINVAL, "n_em must be >= 0");
  if ((r = check_lm(&opts->lm))) return r;
  if (!uvw || !freqs || !V || !jones) return fail(SC_EINVAL, "uvw, freqs, V and jones must not be NULL");
  if ((r = open_ctx(c, d, prec, ws, ws_bytes, stream))) return r;
  const Shape& s = c.s;
  const size_t rs = prec == SC_MIXED ? 4 : 8;
  const size_t v_chunk = (size_t)s.T * s.B * s.F * 8 * rs;   // bytes of one chunk's data
  const size_t u_chunk = (size_t)s.T * s.N * 3;              // doubles of one chunk's uvw
  const size_t j_all = (size_t)s.K * s.N * 8;                // doubles of one Jones set
  for (int i = 0; i < n_chunks; ++i) {
    const void* Vi = static_cast<const char*>(V) + v_chunk * i;
    double* ci = costs ? costs + (size_t)s.K * i : nullptr;
    r = prec == SC_MIXED
            ? sage<float>(c, uvw + u_chunk * i, freqs, sky, static_cast<const float*>(Vi), jones, *opts, ci)
            : sage<double>(c, uvw + u_chunk * i, freqs, sky, static_cast<const double*>(Vi), jones, *opts, ci);
    if (r) return r;
    if (jones_out)
      SC_CUDA(cudaMemcpyAsync(jones_out + j_all * i, jones, j_all * sizeof(double), cudaMemcpyDeviceToDevice,
                              c.st));
  }
  return ok();
}

}  // extern "C"

// A captured sc_calibrate_sage call: the instantiated graph, the device it
// belongs to and the number of library kernels one replay launches.
struct sc_graph {
  cudaGraph_t graph;
  cudaGraphExec_t exec;
  int device;
  unsigned long long kernels;
};

extern "C" {

SC_API int32_t sc_graph_capture_sage(const sc_dims* d, const double* uvw, const double* freqs,
                                     const sc_sky* sky, const void* V, double* jones,
                                     const sc_sage_opts* opts, double* costs, int32_t prec, void* ws,
                                     size_t ws_bytes, void* stream, sc_graph** graph) {
  if (graph == nullptr) return fail(SC_EINVAL, "graph is NULL");
  *graph = nullptr;
  if (stream == nullptr) return fail(SC_EINVAL, "capture needs a created stream, not the legacy default stream");
  if (prof_active()) return fail(SC_EINVAL, "per-kernel profiling is on; call sc_profile_end() before capturing");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  SC_CUDA(cudaStreamIsCapturing(st, &cs));
  if (cs != cudaStreamCaptureStatusNone) return fail(SC_EINVAL, "stream is already capturing");
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  const unsigned long long n0 = launch_count();
  // relaxed: the first call on a device sets kernel attributes and queries
  // occupancy, which are not stream work
  SC_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed));
  const int r = sc_calibrate_sage(d, uvw, freqs, sky, V, jones, opts, costs, prec, ws, ws_bytes, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(st, &g);
  if (r != SC_OK) {  // keeps sc_calibrate_sage's message
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (ee != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    return fail(SC_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ee));
  }
  cudaGraphExec_t ex = nullptr;
  const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    return fail(SC_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
  }
  sc_graph* h = new (std::nothrow) sc_graph{g, ex, dev, launch_count() - n0};
  if (h == nullptr) {
    cudaGraphExecDestroy(ex);
    cudaGraphDestroy(g);
    return fail(SC_ENOMEM, "out of host memory for the graph handle");
  }
  *graph = h;
  return ok();
}

SC_API int32_t sc_graph_launch(sc_graph* graph, void* stream) {
  if (graph == nullptr) return fail(SC_EINVAL, "graph is NULL");
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  if (dev != graph->device)
    return fail(SC_EINVAL, "graph captured on device %d, current device is %d", graph->device, dev);
  SC_CUDA(cudaGraphLaunch(graph->exec, static_cast<cudaStream_t>(stream)));
  count_launches(graph->kernels);
  return ok();
}

SC_API int32_t sc_graph_destroy(sc_graph* graph) {
  if (graph == nullptr) return ok();
  cudaGraphExecDestroy(graph->exec);
  cudaGraphDestroy(graph->graph);
  delete graph;
  return ok();
}

SC_API int32_t sc_calibrate_consensus(const sc_dims* d, int32_t n_bands, const double* uvw,
                                      const double* freqs, const sc_sky* sky, const void* V,
                                      const double* basis, double* jones, double* dual, double* Z,
                                      double* costs, const sc_consensus_opts* opts, int32_t prec,
                                      void* ws, size_t ws_bytes, void* stream) {
  Ctx c;
  // argument checks first: they touch no device memory
  int r = check_dims(d, prec, c.s);
  if (r) return r;
  if (!opts) return fail(SC_EINVAL, "options are NULL");
  if (opts->n_poly < 1 || opts->n_poly > kMaxPoly)
    return fail(SC_EINVAL, "n_poly = %d outside [1, %d]", opts->n_poly, kMaxPoly);
  if (n_bands < opts->n_poly || n_bands > kMaxBands)
    return fail(SC_EINVAL, "n_bands = %d outside [n_poly = %d, %d]", n_bands, opts->n_poly, kMaxBands);
  if (opts->n_admm < 1) return fail(SC_EINVAL, "n_admm must be >= 1");
  if (!(opts->rho >= 0) || !(opts->rho < 1e300)) return fail(SC_EINVAL, "rho must be finite and >= 0");
  if (opts->sage.n_em < 0) return fail(SC_EINVAL, "n_em must be >= 0");
  if ((r = check_lm(&opts->sage.lm))) return r;
  if ((r = check_sky(c.s, sky))) return r;
  if (!uvw || !freqs || !V || !basis || !jones || !dual || !Z)
    return fail(SC_EINVAL, "uvw, freqs, V, basis, jones, dual and Z must not be NULL");
  if ((r = open_ctx(c, d, prec, ws, ws_bytes, stream))) return r;
  const Shape& s = c.s;
  const int P = 8 * s.N, K = s.K, n_poly = opts->n_poly;
  const size_t rs = prec == SC_MIXED ? 4 : 8;
  const size_t v_band = (size_t)s.T * s.B * s.F * 8 * rs;  // bytes of one band's data
  const size_t j_band = (size_t)K * P;                      // doubles of one band's Jones
  const double pen_w = 0.5 * opts->rho;
  // band workspaces: as many whole ones as ws holds, at most one per band
  const size_t per = align256(c.L.total);
  const int m = (int)std::max<size_t>(1, std::min<size_t>({ws_bytes / per, (size_t)n_bands, (size_t)kConsensusStreams}));
  cudaStream_t streams[kConsensusStreams];
  cudaEvent_t fork = nullptr, joins[kConsensusStreams];
  sc_sage_opts so = opts->sage;
  if (m > 1) {
    if ((r = consensus_streams(m, streams, &fork, joins))) return r;
    if (so.lm.max_ctas == 0) so.lm.max_ctas = std::max(8, 2 * device_sms() / m);
  }
  std::vector<Ctx> band(m, c);
  for (int k = 1; k < m; ++k) {
    band[k].base = c.base + per * k;
    SC_CUDA(cudaMemsetAsync(band[k].status(), 0, 256, c.st));
  }
  for (int it = 0; it < opts->n_admm; ++it) {
    if (m > 1) {
      SC_CUDA(cudaEventRecord(fork, c.st));
      for (int k = 0; k < m; ++k) {
        SC_CUDA(cudaStreamWaitEvent(streams[k], fork, 0));
        band[k].st = streams[k];
      }
    }
    for (int f = 0; f < n_bands; ++f) {
      const Ctx& cb = band[f % m];
      double* target = cb.at<double>(cb.L.pen);
      const double* pen = nullptr;
      if (it > 0) {
        SC_CUDA(launch_consensus_target(f, n_poly, K, P, basis, Z, dual, target, cb.st));
        pen = target;
      }
      const void* Vf = static_cast<const char*>(V) + v_band * f;
      double* cf = costs ? costs + (size_t)K * f : nullptr;
      r = prec == SC_MIXED
              ? sage<float>(cb, uvw, freqs + (size_t)s.F * f, sky, static_cast<const float*>(Vf), jones + j_band * f,
                            so, cf, pen, pen_w)
              : sage<double>(cb, uvw, freqs + (size_t)s.F * f, sky, static_cast<const double*>(Vf),
                             jones + j_band * f, so, cf, pen, pen_w);
      if (r) return r;
    }
    if (m > 1) {
      for (int k = 0; k < m; ++k) {
        SC_CUDA(cudaEventRecord(joins[k], streams[k]));
        SC_CUDA(cudaStreamWaitEvent(c.st, joins[k], 0));
      }
    }
    SC_LAUNCH(PK_OTHER, launch_consensus_fit(n_bands, n_poly, K, P, basis, jones, dual, Z, c.status(), c.st));
    SC_LAUNCH(PK_OTHER, launch_consensus_dual(n_bands, n_poly, K, P, basis, jones, Z, dual, c.st));
  }
  for (int k = 1; k < m; ++k) SC_LAUNCH(PK_OTHER, launch_or_status(band[k].status(), c.status(), c.st));
  return ok();
}

SC_API int32_t sc_calibrate_batch(const sc_job* jobs, int32_t n_jobs, const sc_sage_opts* opts, int32_t prec) {
  if (n_jobs < 0 || (n_jobs > 0 && jobs == nullptr)) return fail(SC_EINVAL, "bad job array");
  if (!opts) return fail(SC_EINVAL, "options are NULL");
  if (n_jobs == 0) return ok();
  int dev = 0;
  SC_CUDA(cudaGetDevice(&dev));
  int sms = 152;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  unsigned hw = std::max(1u, std::thread::hardware_concurrency());
  int workers = (int)std::min<unsigned>((unsigned)n_jobs, std::min(hw, 16u));
  sc_sage_opts o = *opts;
  if (o.lm.max_ctas == 0) o.lm.max_ctas = std::max(8, 2 * sms / workers);
  std::atomic<int> next{0};
  std::atomic<int> first_err{0};
  std::vector<std::string> msgs(workers);
  auto work = [&](int wid) {
    cudaSetDevice(dev);
    for (;;) {
      int i = next.fetch_add(1);
      if (i >= n_jobs) break;
      const sc_job& j = jobs[i];
      int r = sc_calibrate_sage(&j.dims, j.uvw, j.freqs, &j.sky, j.V, j.jones, &o, j.costs, prec, j.ws, j.ws_bytes,
                                j.stream);
      if (r != SC_OK) {
        int z = 0;
        if (first_err.compare_exchange_strong(z, r)) {
          char buf[512];
          sc_last_error(buf, sizeof(buf));
          msgs[wid] = std::string("job ") + std::to_string(i) + ": " + buf;
        }
      }
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < workers; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& t : pool) t.join();
  int r = first_err.load();
  if (r != SC_OK) {
    for (auto& m : msgs)
      if (!m.empty()) return fail(r, "%s", m.c_str());
    return fail(r, "a job failed");
  }
  return ok();
}

// checks of a lock-step batch that touch no device memory; T_max of the jobs
static int check_batched(const sc_dims* dims, int32_t n_jobs, int32_t prec, Shape& s0, int& T_max) {
  if (n_jobs < 1 || dims == nullptr) return fail(SC_EINVAL, "a batch needs at least one job");
  T_max = 0;
  for (int g = 0; g < n_jobs; ++g) {
    Shape s;
    if (check_dims(&dims[g], prec, s)) {
      const std::string m = g_msg;
      return fail(SC_EINVAL, "job %d: %s", g, m.c_str());
    }
    if (g == 0) s0 = s;
    else if (s.N != s0.N || s.K != s0.K)
      return fail(SC_EINVAL, "job %d has N = %d, K = %d; a lock-step batch needs the N and K of job 0 (%d, %d)", g,
                  s.N, s.K, s0.N, s0.K);
    T_max = std::max(T_max, s.T);
  }
  return SC_OK;
}

SC_API int32_t sc_batched_workspace_size(const sc_dims* dims, int32_t n_jobs, int32_t prec, size_t* bytes) {
  Shape s0;
  int T_max = 0;
  int r = check_batched(dims, n_jobs, prec, s0, T_max);
  if (r) return r;
  if (!bytes) return fail(SC_EINVAL, "bytes is NULL");
  *bytes = plan_batched(s0, T_max, n_jobs).total;
  return ok();
}

SC_API int32_t sc_calibrate_batched(const sc_job* jobs, int32_t n_jobs, const sc_sage_opts* opts, int32_t prec,
                                    int32_t window, void* ws, size_t ws_bytes, void* stream) {
  if (n_jobs < 1 || jobs == nullptr) return fail(SC_EINVAL, "a batch needs at least one job");
  if (!opts) return fail(SC_EINVAL, "options are NULL");
  if (opts->n_em < 0) return fail(SC_EINVAL, "n_em must be >= 0");
  int r = check_lm(&opts->lm);
  if (r) return r;
  if (opts->lm.chol_kernel != SC_CHOL_SIMT)
    return fail(SC_EINVAL, "the batched factorisation has only the SC_CHOL_SIMT kernel");
  if (window < 0 || window > (1 << 20)) return fail(SC_EINVAL, "window must be in [0, 2^20]");
  std::vector<sc_dims> dims(n_jobs);
  for (int g = 0; g < n_jobs; ++g) dims[g] = jobs[g].dims;
  Shape s0;
  int T_max = 0;
  if ((r = check_batched(dims.data(), n_jobs, prec, s0, T_max))) return r;
  for (int g = 0; g < n_jobs; ++g) {
    const sc_job& j = jobs[g];
    Shape sj;
    check_dims(&j.dims, prec, sj);
    if (check_sky(sj, &j.sky)) {
      const std::string m = g_msg;
      return fail(SC_EINVAL, "job %d: %s", g, m.c_str());
    }
    if (!j.uvw || !j.freqs || !j.V || !j.jones)
      return fail(SC_EINVAL, "job %d: uvw, freqs, V and jones must not be NULL", g);
    if (!j.ws || (reinterpret_cast<uintptr_t>(j.ws) & 255))
      return fail(SC_EINVAL, "job %d: workspace NULL or not 256-byte aligned", g);
    const size_t need = plan_workspace(sj, true).total;
    if (j.ws_bytes < need) return fail(SC_ENOMEM, "job %d: workspace of %zu bytes, %zu needed", g, j.ws_bytes, need);
  }
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(SC_EINVAL, "batch workspace NULL or not 256-byte aligned");
  Ctx c;
  c.s = s0;
  const BatchedLayout bl = plan_batched(s0, T_max, n_jobs);
  c.L = bl.block;
  if (ws_bytes < bl.total) return fail(SC_ENOMEM, "batch workspace of %zu bytes, %zu needed", ws_bytes, bl.total);
  c.base = static_cast<char*>(ws);
  c.st = static_cast<cudaStream_t>(stream);
  c.splits = 1;
  // the batch runs on `stream` after the work already queued on each job's stream
  for (int g = 0; g < n_jobs; ++g) {
    if (jobs[g].stream == stream) continue;
    cudaEvent_t ev = nullptr;
    SC_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    SC_CUDA(cudaEventRecord(ev, static_cast<cudaStream_t>(jobs[g].stream)));
    SC_CUDA(cudaStreamWaitEvent(c.st, ev, 0));
    SC_CUDA(cudaEventDestroy(ev));
  }
  std::vector<Ctx> jc(n_jobs);
  for (int g = 0; g < n_jobs; ++g)
    if ((r = open_ctx(jc[g], &jobs[g].dims, prec, jobs[g].ws, jobs[g].ws_bytes, stream))) return r;
  uint32_t* order = nullptr;  // window 0: the lists interleaved, no table
  if (window > 0) {
    if (!bl.order) return fail(SC_EINVAL, "these jobs are too many or too large for a staggered order");
    order = c.at<uint32_t>(bl.order);
    SC_LAUNCH(PK_OTHER, launch_batch_order(c.L.nT, n_jobs, window, order, c.st));
  }
  r = prec == SC_MIXED ? sage_batched<float>(c, jc, jobs, *opts, order)
                       : sage_batched<double>(c, jc, jobs, *opts, order);
  if (r) return r;
  // each job's stream continues after the batch
  cudaEvent_t done = nullptr;
  SC_CUDA(cudaEventCreateWithFlags(&done, cudaEventDisableTiming));
  SC_CUDA(cudaEventRecord(done, c.st));
  for (int g = 0; g < n_jobs; ++g)
    if (jobs[g].stream != stream) SC_CUDA(cudaStreamWaitEvent(static_cast<cudaStream_t>(jobs[g].stream), done, 0));
  SC_CUDA(cudaEventDestroy(done));
  return ok();
}

SC_API int32_t sc_tune_batched(const sc_dims* dims, int32_t n_jobs, int32_t prec, const int32_t* windows,
                                int32_t n_windows, int32_t reps, double* ms_out, int32_t* best, void* ws,
                                size_t ws_bytes, void* stream) {
  Shape s0;
  int T_max = 0;
  int r = check_batched(dims, n_jobs, prec, s0, T_max);
  if (r) return r;
  if (n_windows < 1 || windows == nullptr || ms_out == nullptr || best == nullptr || reps < 1)
    return fail(SC_EINVAL, "windows, ms_out and best must not be NULL, n_windows and reps >= 1");
  for (int i = 0; i < n_windows; ++i)
    if (windows[i] < 1 || windows[i] > (1 << 20))
      return fail(SC_EINVAL, "window %d is %d; windows must be in [1, 2^20]", i, windows[i]);
  if (ws == nullptr || (reinterpret_cast<uintptr_t>(ws) & 255))
    return fail(SC_EINVAL, "batch workspace NULL or not 256-byte aligned");
  const BatchedLayout bl = plan_batched(s0, T_max, n_jobs);
  if (ws_bytes < bl.total) return fail(SC_ENOMEM, "batch workspace of %zu bytes, %zu needed", ws_bytes, bl.total);
  if (!bl.order) return fail(SC_EINVAL, "these jobs are too many or too large for a staggered order");
  Ctx c;
  c.s = s0;
  c.L = bl.block;
  c.base = static_cast<char*>(ws);
  c.st = static_cast<cudaStream_t>(stream);
  c.splits = 1;
  const Workspace& L = c.L;
  const size_t js = L.total;
  const Batch bt{n_jobs, js};
  const size_t rs = prec == SC_MIXED ? 4 : 8;
  // identity matrices (the arithmetic takes the same time on any values),
  // LM states that are not done, clear status words
  SC_CUDA(cudaMemset2DAsync(c.base + L.A, js, 0, (size_t)L.Ppad * L.Ppad * rs, n_jobs, c.st));
  SC_CUDA(cudaMemset2DAsync(c.base + L.lm, js, 0, sizeof(LMState), n_jobs, c.st));
  SC_CUDA(cudaMemset2DAsync(c.base + L.status, js, 0, 256, n_jobs, c.st));
  for (int g = 0; g < n_jobs; ++g) {
    char* A = c.base + (size_t)g * js + L.A;
    if (prec == SC_MIXED) SC_CUDA(launch_pad_identity(reinterpret_cast<float*>(A), L.Ppad, 0, c.st));
    else SC_CUDA(launch_pad_identity(reinterpret_cast<double*>(A), L.Ppad, 0, c.st));
  }
  uint32_t* order = c.at<uint32_t>(bl.order);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  SC_CUDA(cudaEventCreate(&e0));
  SC_CUDA(cudaEventCreate(&e1));
  auto factor = [&]() -> cudaError_t {
    return prec == SC_MIXED
               ? launch_chol_batch<float>(c.at<float>(L.A), L.Ppad, L.nT, c.at<float>(L.Linv), c.at<int>(L.sync),
                                          c.status(), c.lm(), 0, bt, order, c.st)
               : launch_chol_batch<double>(c.at<double>(L.A), L.Ppad, L.nT, c.at<double>(L.Linv),
                                           c.at<int>(L.sync), c.status(), c.lm(), 0, bt, order, c.st);
  };
  int bi = 0;
  cudaError_t e = cudaSuccess;
  for (int i = 0; i < n_windows && e == cudaSuccess; ++i) {
    const int W = windows[i];
    // each run factorises identities again: the factor of I is I
    if ((e = launch_batch_order(L.nT, n_jobs, W, order, c.st)) != cudaSuccess) break;
    if ((e = factor()) != cudaSuccess) break;  // warm-up
    if ((e = cudaEventRecord(e0, c.st)) != cudaSuccess) break;
    for (int k = 0; k < reps && e == cudaSuccess; ++k) e = factor();
    if (e != cudaSuccess || (e = cudaEventRecord(e1, c.st)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    ms_out[i] = ms / reps;
    if (ms_out[i] < ms_out[bi]) bi = i;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return fail(SC_ECUDA, "tuning the batched factorisation: %s", cudaGetErrorString(e));
  *best = windows[bi];
  return ok();
}

SC_API int32_t sc_batch_order(int32_t nT, int32_t n_jobs, int32_t window, int32_t* out, int64_t cap) {
  if (nT < 1 || n_jobs < 1 || window < 1 || window > (1 << 20) || !batch_order_ok(nT, n_jobs) || out == nullptr)
    return fail(SC_EINVAL, "bad batch order arguments");
  const int n = chol_ntasks(nT);
  if (cap < (int64_t)n * n_jobs) return fail(SC_EINVAL, "out holds %lld entries, %lld needed", (long long)cap,
                                              (long long)n * n_jobs);
  for (int g = 0; g < n_jobs; ++g)
    for (int t = 0; t < n; ++t) out[(size_t)g * n + t] = batch_order_pos(n, n_jobs, window, g, t);
  return ok();
}

}  // extern "C"
