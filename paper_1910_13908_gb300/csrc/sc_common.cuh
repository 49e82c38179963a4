// Shared device helpers: 2x2 complex algebra, baseline indexing, the device
// LM state and the internal launcher declarations of every kernel file.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/sagecal_gb.h"

namespace sc {

constexpr double kCLight = 299792458.0;
constexpr int kNB = 64;          // Cholesky tile edge
constexpr int kCholThreads = 256;
constexpr int kMaxParts = 4096;  // per-block partial sums of sc_residual_all
constexpr int kMaxSMs = 512;     // multiprocessor count the workspace layout allows for

// ---- complex scalars -----------------------------------------------------------

template <typename R> struct Vec2;
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<double> { using T = double2; };

template <typename R>
struct cx {
  R re, im;
};

template <typename R> __host__ __device__ __forceinline__ cx<R> cmk(R a, R b) { return {a, b}; }
template <typename R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cx<R> conj(cx<R> a) { return {a.re, -a.im}; }
template <typename R> __device__ __forceinline__ cx<R> scale(cx<R> a, R s) { return {a.re * s, a.im * s}; }
// conj(a) * b
template <typename R> __device__ __forceinline__ cx<R> cmulc(cx<R> a, cx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}
template <typename R> __device__ __forceinline__ R norm2(cx<R> a) { return a.re * a.re + a.im * a.im; }

// ---- 2x2 complex matrices, row-major (a b; c d) ------------------------------------

template <typename R>
struct m22 {
  cx<R> a, b, c, d;
};

template <typename R> __device__ __forceinline__ m22<R> operator+(const m22<R>& x, const m22<R>& y) {
  return {x.a + y.a, x.b + y.b, x.c + y.c, x.d + y.d};
}
template <typename R> __device__ __forceinline__ m22<R> operator-(const m22<R>& x, const m22<R>& y) {
  return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d};
}
template <typename R> __device__ __forceinline__ m22<R> smul(cx<R> s, const m22<R>& x) {
  return {s * x.a, s * x.b, s * x.c, s * x.d};
}
// x * y
template <typename R> __device__ __forceinline__ m22<R> mul(const m22<R>& x, const m22<R>& y) {
  return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
// x * y^H
template <typename R> __device__ __forceinline__ m22<R> mul_h(const m22<R>& x, const m22<R>& y) {
  return {x.a * conj(y.a) + x.b * conj(y.b), x.a * conj(y.c) + x.b * conj(y.d),
          x.c * conj(y.a) + x.d * conj(y.b), x.c * conj(y.c) + x.d * conj(y.d)};
}
// x^H * y
template <typename R> __device__ __forceinline__ m22<R> h_mul(const m22<R>& x, const m22<R>& y) {
  return {cmulc(x.a, y.a) + cmulc(x.c, y.c), cmulc(x.a, y.b) + cmulc(x.c, y.d),
          cmulc(x.b, y.a) + cmulc(x.d, y.c), cmulc(x.b, y.b) + cmulc(x.d, y.d)};
}
template <typename R> __device__ __forceinline__ m22<R> hconj(const m22<R>& x) {
  return {conj(x.a), conj(x.c), conj(x.b), conj(x.d)};
}
template <typename R> __device__ __forceinline__ R frob2(const m22<R>& x) {
  return norm2(x.a) + norm2(x.b) + norm2(x.c) + norm2(x.d);
}
template <typename R> __device__ __forceinline__ m22<R> mzero() {
  return {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
}

// Jones of station s from the float64 parameter vector (8 doubles).
template <typename R>
__device__ __forceinline__ m22<R> load_jones(const double* __restrict__ J, int s) {
  const double2* p = reinterpret_cast<const double2*>(J + 8 * s);
  double2 a = p[0], b = p[1], c = p[2], d = p[3];
  return {{(R)a.x, (R)a.y}, {(R)b.x, (R)b.y}, {(R)c.x, (R)c.y}, {(R)d.x, (R)d.y}};
}

// ---- visibility element loads / stores (one 2x2 complex) ---------------------------

__device__ __forceinline__ m22<float> ld_vis(const float* __restrict__ p) {
  float4 u = __ldg(reinterpret_cast<const float4*>(p));
  float4 v = __ldg(reinterpret_cast<const float4*>(p) + 1);
  return {{u.x, u.y}, {u.z, u.w}, {v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ m22<double> ld_vis(const double* __restrict__ p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  return {{a.x, a.y}, {b.x, b.y}, {c.x, c.y}, {d.x, d.y}};
}
__device__ __forceinline__ void st_vis(float* p, const m22<float>& x) {
  reinterpret_cast<float4*>(p)[0] = make_float4(x.a.re, x.a.im, x.b.re, x.b.im);
  reinterpret_cast<float4*>(p)[1] = make_float4(x.c.re, x.c.im, x.d.re, x.d.im);
}
__device__ __forceinline__ void st_vis(double* p, const m22<double>& x) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(x.a.re, x.a.im);
  q[1] = make_double2(x.b.re, x.b.im);
  q[2] = make_double2(x.c.re, x.c.im);
  q[3] = make_double2(x.d.re, x.d.im);
}
__device__ __forceinline__ cx<float> ld_c(const float* __restrict__ p) {
  float2 u = __ldg(reinterpret_cast<const float2*>(p));
  return {u.x, u.y};
}
__device__ __forceinline__ cx<double> ld_c(const double* __restrict__ p) {
  double2 u = __ldg(reinterpret_cast<const double2*>(p));
  return {u.x, u.y};
}

// ---- baselines -----------------------------------------------------------------------

__host__ __device__ __forceinline__ int64_t row_start(int p, int N) {
  return (int64_t)p * N - (int64_t)p * (p + 1) / 2;
}
__host__ __device__ __forceinline__ int64_t bl_index(int p, int q, int N) {
  return row_start(p, N) + (q - p - 1);
}
// inverse of bl_index: a float32 estimate from the quadratic formula (FP32
// is 64x the FP64 rate here), made exact by the integer comparisons below
__device__ __forceinline__ void bl_pair(int64_t b, int N, int& p, int& q) {
  const float n2 = 2.0f * N - 1.0f;
  int pp = (int)floorf(0.5f * (n2 - sqrtf(fmaxf(n2 * n2 - 8.0f * (float)b, 0.0f))));
  if (pp < 0) pp = 0;
  if (pp > N - 2) pp = N - 2;
  while (pp > 0 && row_start(pp, N) > b) --pp;
  while (pp < N - 2 && row_start(pp + 1, N) <= b) ++pp;
  p = pp;
  q = (int)(b - row_start(pp, N)) + pp + 1;
}

// ---- device LM state ---------------------------------------------------------------

struct LMState {
  double mu, nu;
  double cost, cost_trial, pred, rho;
  double lm_tau, eps_grad;
  int32_t iter, n_lm, done, notpd, skip, accepted;
  int32_t nchunk;  // timeslot chunks of the statistics (set by the statistics pass of a batched solve)
  int32_t pad;
};

// Device buffers of one LM solve's state: current and trial Jones,
// J^T r, diagonal blocks H, station costs and per-station maxima of |J^T r|;
// the trial step's partial predicted decreases; in float32 the Jones rounded
// once for the J^T J assembly (NULL in float64).
struct LMBufs {
  double *J_cur, *J_trial, *g_cur, *g_trial, *H_cur, *H_trial, *cp_cur, *cp_trial, *gm_cur, *gm_trial;
  double* pred_part;
  float *Jf_cur, *Jf_trial;
};

// A lock-step batch: G jobs of equal station count whose LM buffers lie at a
// fixed byte stride js from those of job 0.  Each launch covers every job;
// a kernel takes its job from blockIdx.z (the persistent factorisation and
// the solves from the task index) and moves every buffer pointer by
// job * js.  G = 1, js = 0 is a single solve.
struct Batch {
  int G = 1;
  size_t js = 0;
};
template <typename T>
__host__ __device__ __forceinline__ T* job_ptr(T* p, size_t js, int g) {
  return p == nullptr ? p : reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + (size_t)g * js);
}
__host__ __device__ __forceinline__ LMBufs job_bufs(LMBufs b, size_t js, int g) {
  return {job_ptr(b.J_cur, js, g),   job_ptr(b.J_trial, js, g),  job_ptr(b.g_cur, js, g),
          job_ptr(b.g_trial, js, g), job_ptr(b.H_cur, js, g),    job_ptr(b.H_trial, js, g),
          job_ptr(b.cp_cur, js, g),  job_ptr(b.cp_trial, js, g), job_ptr(b.gm_cur, js, g),
          job_ptr(b.gm_trial, js, g), job_ptr(b.pred_part, js, g), job_ptr(b.Jf_cur, js, g),
          job_ptr(b.Jf_trial, js, g)};
}

// ---- workspace ------------------------------------------------------------------------

// Offsets of every scratch buffer inside the caller's workspace.
struct Workspace {
  size_t total;
  // always present
  size_t status;     // uint32 device status word (+ padding)
  size_t lm;         // LMState
  // job-level buffers
  size_t C;          // [K][T][B][F] complex  (SAGE only)
  size_t w;          // [K][B] real
  size_t wpart;      // [splits][B] real (predict partial sums)
  size_t Rres;       // [T][B][F][4] complex running residual (SAGE only)
  size_t E;          // [T][F][S_max][N] float2 station phasors (mixed)
  size_t Sf;         // [F][S_max] float fluxes at each channel (mixed)
  // per-solve buffers
  size_t stat_cost;  // [nchunk][B] real
  size_t stat_rho;   // [nchunk][B][8] real
  size_t lstat;      // [nchunk][10][B] double: per-baseline statistics of an LM solve
  size_t part;       // per-tile partials of an LM evaluation (double)
  size_t J_old, J_cur, J_trial;  // [8N] double
  size_t g_cur, g_trial;         // [8N] double
  size_t H_cur, H_trial;         // [4N] double
  size_t cpart_cur, cpart_trial; // [N] double
  size_t gm_cur, gm_trial;       // [N] double, max_i |J^T r| of each station
  size_t pred_part;              // [8N / 256 + 1] double, partial predicted decreases
  size_t Jf_cur, Jf_trial;       // [8N] float, the Jones rounded for the float32 assembly
  size_t x, rvec, ry;            // [Ppad] double (ry: X_o^H J_o of the refinement)
  size_t bvec;                   // [Ppad] solved blocks as tagged 64-bit words (1 per float, 2 per double)
  size_t A;          // [Ppad][Ppad] real
  size_t Linv;       // [nT][64][64] real
  size_t sync;       // int: task counters, tile counters, flags
  // residual of all clusters (sc_residual_all)
  size_t gains;      // [K][N][8] real, every cluster's Jones rounded to the data type
  size_t gain_inv;   // [N][8] real, inverse Jones of the correction direction
  size_t parts;      // [kMaxParts] double, per-block cost sums
  // polarised prediction (sc_predict_coherencies_full)
  size_t srcp;       // [2][F][S_max] float4: spectral Stokes, Gaussian quadratic form
  // consensus across sub-bands (sc_calibrate_consensus)
  size_t pen;        // [K][8N] double, penalty targets of one band's clusters
  int nT, Ppad, nchunk, tchunk, splits;
};

struct Shape {
  int N, T, F, K, S_max;
  int64_t B;
  int prec;  // SC_FP64 / SC_MIXED
};

// computes the layout; `job` = true to include the SAGE job buffers
Workspace plan_workspace(const Shape& s, bool job);

// ---- opt-in kernel timing (prof.cu) ---------------------------------------------------------

enum ProfKind {
  PK_PHASORS = 0,   // station phasors (mixed predict)
  PK_COHERENCY,     // coherency contraction (mixed) / direct predict (FP64)
  PK_PASS,          // streaming pass over the visibilities
  PK_REDUCE,        // per-station reduction
  PK_ASSEMBLE,      // J^T J assembly
  PK_CHOL,          // Cholesky factorisation
  PK_SOLVE,         // triangular solves
  PK_REFINE,        // float64 refinement residual
  PK_LM,            // LM control
  PK_OTHER,         // small helpers (w sums, cost sums)
  PK_STATS,         // per-baseline statistics of an LM solve (one pass over the data)
  PK_COUNT
};
void prof_start(int kind, cudaStream_t st);
void prof_stop(int kind, cudaStream_t st);  // also counts the launch
unsigned long long launch_count();
void count_launches(unsigned long long n);  // kernels launched by a graph replay
bool prof_active();
int prof_begin();
int prof_end();
void prof_read(int kind, long* n, double* ms);

// ---- launchers (internal; all asynchronous on `st`) -------------------------------------

// one cluster of a polarised sky (device pointers at its first source)
struct SkyFull {
  const double *l, *m, *I, *Q, *U, *V, *alpha, *maj, *mnr, *pa;
  double f0;
};

// consensus.cu: the Z-step, the penalty targets and the dual step of the
// consensus across sub-bands; basis [n_bands][n_poly], Jones and duals
// [n_bands][K][8N], Z [K][n_poly][8N] (all float64, device)
constexpr int kMaxBands = 256;
constexpr int kMaxPoly = 8;
cudaError_t launch_consensus_fit(int n_bands, int n_poly, int K, int P, const double* basis,
                                 const double* J, const double* U, double* Z, uint32_t* status,
                                 cudaStream_t st);
cudaError_t launch_consensus_target(int band, int n_poly, int K, int P, const double* basis,
                                    const double* Z, const double* U, double* target, cudaStream_t st);
cudaError_t launch_consensus_dual(int n_bands, int n_poly, int K, int P, const double* basis,
                                  const double* J, const double* Z, double* U, cudaStream_t st);
cudaError_t launch_or_status(const uint32_t* src, uint32_t* dst, cudaStream_t st);

// predict_full.cu
cudaError_t launch_source_params(const Shape& s, int S, const double* freqs, const SkyFull& k, float4* st,
                                 float4* gq, cudaStream_t stream);
cudaError_t launch_coherency_full_f32(const Shape& s, int S, const double* uvw, const float2* E,
                                      const float4* st, const float4* gq, float* C, cudaStream_t stream);
cudaError_t launch_predict_full_f64(const Shape& s, int S, const double* uvw, const double* freqs,
                                    const SkyFull& k, double* C, cudaStream_t stream);

// predict.cu
cudaError_t launch_station_phasors(const Shape& s, const double* uvw, const double* freqs,
                                   const double* l, const double* m, const double* flux,
                                   const double* alpha, double f0, int S, float2* E, float* Sf,
                                   cudaStream_t st);
cudaError_t launch_coherency_f32(const Shape& s, int S, const float2* E, const float* Sf,
                                 float2* C, float* wpart, int splits, cudaStream_t st);
cudaError_t launch_predict_f64(const Shape& s, const double* uvw, const double* freqs,
                               const double* l, const double* m, const double* flux,
                               const double* alpha, double f0, int S, double2* C,
                               cudaStream_t st);
template <typename R>
cudaError_t launch_w_from_C(const Shape& s, const R* C, R* w, cudaStream_t st);
cudaError_t launch_sum_parts(const float* wpart, int splits, int64_t B, float* w, cudaStream_t st);

// lm_pass.cu
enum PassFlags { P_OLD = 1, P_SUB = 2, P_WRITE_R = 4, P_STATS = 8 };
template <typename R>
cudaError_t launch_pass(const Shape& s, int flags, const R* Xin, const R* C, const double* J_old,
                        const double* J_cur, R* Rout, R* stat_cost, R* stat_rho, int nchunk,
                        int tchunk, const LMState* lm, cudaStream_t st);
// lm_stats.cu: the LM loop from per-baseline statistics.  launch_lm_stats
// forms, once per solve, S = sum |X|^2, rhoX = sum conj(c) X and
// W = sum |c|^2 per baseline of the data X = Xin (+ c J_old,p J_old,q^H if
// J_old is not NULL) into stat [nchunk][10][B]; launch_lm_eval then forms,
// per LM evaluation at J, the per-tile partials of the cost, J^T r and H
// (G = J_p J_q^H subtracted if sub, else the residual is X itself), and
// launch_station_sum adds them into g [8N], H [4N] and the station costs
// cpart [N] (and the per-station maxima of |J^T r|, gmax [N]), plus the
// penalty pen_w |theta - pen|^2 if pen is not NULL.
// nchunk_dev, if not NULL, also receives the chunk count on the device.
// In a batch, launch_lm_eval reads each job's chunk count from nchunk_dev
// (moved by the job stride) when it is not NULL, else takes nchunk.
template <typename R>
cudaError_t launch_lm_stats(const Shape& s, const R* Xin, const R* C, const double* J_old, double* stat,
                            int* nchunk, cudaStream_t st, int* nchunk_dev = nullptr);
template <typename R>
cudaError_t launch_lm_eval(const Shape& s, bool sub, const double* stat, int nchunk, const double* J, double* part,
                           const LMState* lm, cudaStream_t st, const Batch& bt = Batch{},
                           const int* nchunk_dev = nullptr);
cudaError_t launch_station_sum(const Shape& s, const double* part, const double* J, double* g, double* H,
                               double* cpart, double* gmax, const LMState* lm, const double* pen, double pen_w,
                               cudaStream_t st, const Batch& bt = Batch{});
size_t lm_stats_doubles(int T, int64_t B);  // size of stat for any GPU of at most kMaxSMs SMs
size_t lm_part_doubles(int N);              // size of the per-tile partials
cudaError_t launch_sum_cost(const double* cpart, int N, double* out, cudaStream_t st);
template <typename R>
cudaError_t launch_sum_reals(const R* x, int64_t n, double* out, cudaStream_t st);

// residual_all.cu
template <typename R>
cudaError_t launch_gain_prep(const Shape& s, const double* J, int corr, R* Jr, R* Jinv,
                             uint32_t* status, cudaStream_t st);
// Jinv = NULL: no correction; part = NULL: no cost partial sums.  Writes the
// number of partial sums (the grid) to *n_parts; at most max_parts.
template <typename R>
cudaError_t launch_residual_all(const Shape& s, const R* V, const R* C, const R* Jr,
                                const R* Jinv, R* Rout, double* part, int max_parts, int* n_parts,
                                cudaStream_t st);

// normal_eqs.cu
// J: the Jones in the matrix's type (rounded once in float32)
template <typename R>
cudaError_t launch_assemble(const Shape& s, int lda, int Ppad, const R* w, const R* J,
                            const double* H, const LMState* lm, R* A, bool damp, bool full,
                            cudaStream_t st, const Batch& bt = Batch{});
cudaError_t launch_round_jones(const double* J, float* Jf, int n, cudaStream_t st);
// r = g - (J^T J + mu I) x in float64; Y [8N] is scratch
template <typename R>
cudaError_t launch_refine_residual(const Shape& s, const R* w, const double* J, const double* H,
                                   const double* g, const double* x, const LMState* lm,
                                   double* Y, double* r, cudaStream_t st, const Batch& bt = Batch{});

// normal_eqs.cu: identity on rows n..Ppad-1 of a zeroed padded matrix
template <typename R>
cudaError_t launch_pad_identity(R* A, int Ppad, int n, cudaStream_t st);

// cholesky.cu
__host__ __device__ int4 chol_task(int nT, int t);   // (type, i, k, j), type -1 past the end
__host__ __device__ int4 solve_task(int nT, int t);
int chol_ntasks(int nT);
int chol_sync_ints(int nT);
// kernel: SC_CHOL_SIMT or SC_CHOL_TENSOR (float32 only)
template <typename R>
cudaError_t launch_chol(R* A, int lda, int nT, R* Linv, int* sync, uint32_t* status, LMState* lm,
                        int max_ctas, int kernel, cudaStream_t st);
// The factorisations of a whole batch as one persistent launch: the task
// lists of the G jobs interleaved (task t is task t / G of job t mod G), no
// walker; every tile is computed by the same arithmetic as in launch_chol.
template <typename R>
cudaError_t launch_chol_batch(R* A, int lda, int nT, R* Linv, int* sync, uint32_t* status, LMState* lm,
                              int max_ctas, const Batch& bt, const uint32_t* order, cudaStream_t st);
// The combined task order of a batch with the jobs staggered over a window
// of W jobs: entry m is job << 20 | task (order [G * chol_ntasks(nT)]).
// Possible when batch_order_ok (G <= 4096, at most 2^20 tasks per job);
// otherwise the factorisation interleaves the lists (order NULL).
__host__ __device__ int batch_order_pos(int n, int G, int W, int g, int t);
bool batch_order_ok(int nT, int G);
cudaError_t launch_batch_order(int nT, int G, int W, uint32_t* order, cudaStream_t st);
template <typename R>
cudaError_t launch_chol_solve(const R* A, int lda, int nT, const R* Linv, int* sync,
                              const double* b, uint64_t* bwork, double* x, int accumulate,
                              uint32_t* status, const LMState* lm, cudaStream_t st, const Batch& bt = Batch{});

// lm_control.cu
cudaError_t launch_lm_init(LMState* lm, const sc_lm_opts* o, int N, const LMBufs& b, const double* J_src,
                           cudaStream_t st, const Batch& bt = Batch{});
cudaError_t launch_lm_trial(LMState* lm, int N, const double* x, const LMBufs& b, cudaStream_t st,
                            const Batch& bt = Batch{});
int lm_trial_blocks(int N);
cudaError_t launch_lm_decide(LMState* lm, int N, const LMBufs& b, cudaStream_t st, const Batch& bt = Batch{});
cudaError_t launch_lm_finish(const LMState* lm, const double* J_cur, int N, double* J_out,
                             double* cost_out, int32_t* iters_out, cudaStream_t st);

}  // namespace sc
