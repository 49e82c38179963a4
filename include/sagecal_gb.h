/*
 * sagecal_gb.h -- C ABI of the GB300 SAGE/EM direction-dependent calibration
 * hot path (Spreeuw, van Werkhoven, Yatawatta & Diblen, "GPU acceleration of
 * the SAGECal calibration package for the SKA", arXiv:1910.13908).
 *
 * The paper times SAGECal calibrating a sky model grouped into clusters, one
 * solution per cluster (paper §2), on arrays of N stations whose data grow as
 * the N(N-1)/2 baselines (§3).  The arithmetic it times is SAGECal's:
 *
 *   measurement equation   V_pq = sum_k J_kp C_kpq J_kq^H + noise
 *   point-source coherency C_pq(t,f) = sum_s S_s(f)
 *                              exp(-2 pi i f/c (u l_s + v m_s + w (n_s - 1))) Id
 *   per cluster            Levenberg-Marquardt on the normal equations
 *                          (J^T J + mu I) d = J^T r, solved by a dense
 *                          Cholesky factorisation (8N x 8N)
 *   across clusters        SAGE/EM: each cluster solved in turn against the
 *                          data minus the other clusters' current models.
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Baselines b = (p, q), p < q, b = p*N - p(p+1)/2 + (q-p-1); B = N(N-1)/2.
 *    Autocorrelations are not stored; the q<p baseline is the Hermitian
 *    conjugate of the p<q one.
 *  - Station coordinates uvw: float64 [T][N][3] metres; the (u,v,w) of
 *    baseline pq is uvw_p - uvw_q.
 *  - Visibilities (V, X, R): [T][B][F][2][2] complex, row-major 2x2
 *    (XX, XY, YX, YY), interleaved (re, im): complex64 for SC_MIXED,
 *    complex128 for SC_FP64.
 *  - Coherencies C: [T][B][F] complex (same element type as the
 *    visibilities).  The brightness of an unpolarised point source is a
 *    multiple of the identity, so one complex number per (t, b, f) is the
 *    whole 2x2 coherency c * Id.
 *  - Jones: complex128 [N][2][2] per cluster (always FP64: it is the solver
 *    state); the 8 real parameters of station s are
 *    theta[8s + 4i + 2j + 0/1] = Re/Im J_s[i][j], which is exactly the
 *    memory order of the complex128 array.
 *  - J^T J: [8N][8N] row-major, float (SC_MIXED) or double (SC_FP64);
 *    J^T r: double [8N], with r = X - model, so the LM step solves
 *    (J^T J + mu I) d = J^T r.
 *
 * Memory and streams
 * ------------------
 *  All array pointers are DEVICE pointers owned by the caller unless marked
 *  HOST.  The library allocates no device memory: every call that needs
 *  scratch takes a caller-owned device workspace (ws, ws_bytes) of at least
 *  sc_workspace_size() bytes, 256-byte aligned (sc_residual_noalloc uses a
 *  fixed array compiled into the library instead; a captured graph,
 *  sc_graph_capture_sage, holds host-side driver resources until it is
 *  destroyed).  Every compute call is
 *  asynchronous on `stream` (a cudaStream_t, NULL = legacy default stream);
 *  outputs are valid once the stream has reached that point.  Calls that
 *  share one workspace must not overlap on the device.
 *
 * Errors
 * ------
 *  Every call returns SC_OK (0) or a negative SC_E* code, with a message
 *  retrievable by sc_last_error() (thread-local).  Argument errors are
 *  detected on the host before anything is launched.  Conditions found on
 *  the device (a non-positive-definite damped matrix, a bounded wait that
 *  gave up) are recorded in a status word inside the workspace and returned
 *  by sc_device_status() after the stream has been synchronised.  No call
 *  throws, traps or aborts.
 */
#ifndef SAGECAL_GB_H
#define SAGECAL_GB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SC_API __attribute__((visibility("default")))
#else
#define SC_API
#endif

#define SC_OK 0
#define SC_EINVAL (-1)   /* bad shape, null pointer, N < 2, unknown precision */
#define SC_ENOMEM (-2)   /* workspace smaller than sc_workspace_size() */
#define SC_ENOTPD (-3)   /* damped J^T J not positive definite (device status) */
#define SC_ETIMEOUT (-4) /* a bounded device wait gave up (device status) */
#define SC_ECUDA (-5)    /* a CUDA runtime call failed */

/* Device status bits (sc_device_status) */
#define SC_STATUS_NOTPD 1u
#define SC_STATUS_TIMEOUT 2u
#define SC_STATUS_SINGULAR 4u /* sc_residual_all: a Jones of the correction
                                 direction was singular; its baselines were
                                 zeroed */
#define SC_STATUS_BASIS 8u    /* sc_calibrate_consensus: the normal matrix of
                                 the frequency basis was singular; Z was set
                                 to zero */

typedef enum sc_precision {
  SC_FP64 = 0,  /* everything in float64 / complex128 */
  SC_MIXED = 1  /* float32 data and factorisation, float64 phase argument,
                   float64 Jones state and iterative refinement of the step */
} sc_precision;

/* Shape of one calibration job (one sub-band x time chunk). */
typedef struct sc_dims {
  int32_t N;     /* stations, >= 2 */
  int32_t T;     /* timeslots, >= 1 */
  int32_t F;     /* channels, >= 1 */
  int32_t K;     /* clusters (calibration directions), >= 1 */
  int32_t S_max; /* most sources in any one cluster (>= 1 for calls that predict) */
} sc_dims;

/* Clustered point-source sky model (paper §2: contiguous sources grouped
 * into clusters).  Sources of cluster k are [offsets[k], offsets[k+1]). */
typedef struct sc_sky {
  const int32_t* offsets; /* HOST [K+1], offsets[0] = 0, non-decreasing */
  const double* l;        /* DEVICE [S_total] direction cosine towards east */
  const double* m;        /* DEVICE [S_total] direction cosine towards north */
  const double* flux;     /* DEVICE [S_total] Stokes I flux density at f0, Jy */
  const double* alpha;    /* DEVICE [S_total] spectral index, S(f) = flux (f/f0)^alpha */
  double f0;              /* reference frequency, Hz */
} sc_sky;

/* Clustered sky model of polarised, possibly extended sources (SAGECal's
 * sky models hold full Stokes and Gaussian sources besides points; the
 * paper, §2, groups the sources of a model into clusters).  Sources of
 * cluster k are [offsets[k], offsets[k+1]).  Each DEVICE array holds
 * S_total float64 values. */
typedef struct sc_sky_full {
  const int32_t* offsets; /* HOST [K+1], offsets[0] = 0, non-decreasing */
  const double* l;        /* direction cosine towards east */
  const double* m;        /* direction cosine towards north */
  const double* I;        /* Stokes I at f0, Jy */
  const double* Q;        /* Stokes Q at f0, Jy */
  const double* U;        /* Stokes U at f0, Jy */
  const double* V;        /* Stokes V at f0, Jy */
  const double* alpha;    /* spectral index of all four: S(f) = S (f/f0)^alpha */
  const double* maj;      /* Gaussian FWHM along the major axis, radians (0: point) */
  const double* mnr;      /* Gaussian FWHM along the minor axis, radians (0: point) */
  const double* pa;       /* position angle of the major axis, radians, from
                             +m (north) towards +l (east) */
  double f0;              /* reference frequency, Hz */
} sc_sky_full;

/* Levenberg-Marquardt options (Madsen, Nielsen & Tingleff 2004, Alg. 3.16:
 * damping mu I, mu0 = tau max diag(J^T J), gain-ratio update of mu). */
typedef struct sc_lm_opts {
  int32_t n_lm;          /* trial steps per solve, accepted or rejected */
  int32_t refine_sweeps; /* SC_MIXED: float64 iterative-refinement sweeps of
                            each float32 Cholesky solve (ignored for SC_FP64) */
  double tau;            /* mu0 = tau * max diag(J^T J) */
  double eps_grad;       /* stop once max|J^T r| <= eps_grad * (1 + cost) */
  int32_t max_ctas;      /* cap on the thread blocks of the persistent
                            factorisation kernel; 0 = enough to fill the GPU.
                            Lower it when several jobs share the device. */
  int32_t chol_kernel;   /* SC_MIXED: which factorisation kernel runs the
                            64x64 tile products of the bulk,
                            SC_CHOL_SIMT (0, the default) or SC_CHOL_TENSOR
                            (1); ignored for SC_FP64 */
} sc_lm_opts;

/* Factorisation kernels of the float32 path.  SC_CHOL_SIMT: tile products
 * on the float32 pipes.  SC_CHOL_TENSOR: the TRSM and UPDATE tile products
 * on the tensor cores (tcgen05, operands staged by TMA, three TF32 passes,
 * about 2^-21 relative error per product against 2^-24); the diagonal
 * tiles stay on the float32 pipes.  At the orders of this path the
 * factorisation is bound by the latency of its task graph, not by
 * arithmetic, and the SIMT kernel is the faster of the two. */
#define SC_CHOL_SIMT 0
#define SC_CHOL_TENSOR 1

typedef struct sc_sage_opts {
  int32_t n_em; /* SAGE/EM sweeps over all clusters */
  sc_lm_opts lm;
} sc_sage_opts;

/* Library version, (major << 16) | minor. */
SC_API int32_t sc_version(void);

/* Copies the calling thread's last error message into buf (NUL-terminated,
 * truncated to len).  Returns the last error code. */
SC_API int32_t sc_last_error(char* buf, size_t len);

/* Bytes of device workspace that every call below needs for shape d at
 * precision prec (SC_FP64 / SC_MIXED).  Writes *bytes. */
SC_API int32_t sc_workspace_size(const sc_dims* d, int32_t prec, size_t* bytes);

/* After synchronising the stream of the last call that used ws: the device
 * status word (SC_STATUS_* bits, 0 = clean) of that workspace, which is
 * cleared by every call that launches work on it. */
SC_API int32_t sc_device_status(const void* ws, size_t ws_bytes, uint32_t* status);

/* Diagnostic, host only (launches nothing): the task order of the tiled
 * Cholesky factorisation (which = 0) or of the two triangular solves
 * (which = 1) on an nT x nT grid of 64x64 tiles, as (type, i, k, j)
 * quadruples written to out[0 .. 4*cap).  Types: 0 POTRF(j), 1 TRSM(i, j),
 * 2 UPDATE(i, k, j), 3 forward solve of tile row i, 4 backward solve of tile
 * row i.  With out = NULL only counts.  Returns the number of tasks, or a
 * negative SC_E* code. */
SC_API int32_t sc_chol_schedule(int32_t nT, int32_t which, int32_t* out, int32_t cap);

/* Diagnostics.  sc_launch_count: kernels launched by this library since it
 * was loaded (all threads).  sc_profile_begin / sc_profile_end: while
 * profiling is on, every kernel launch is bracketed by two CUDA events on its
 * stream (a few microseconds each); sc_profile_end waits for them and
 * sc_profile_read returns, per kernel kind, the launches and their summed
 * device time in ms.  Kinds: 0 station phasors, 1 coherency contraction /
 * FP64 direct predict, 2 visibility pass, 3 station reduction, 4 J^T J
 * assembly, 5 Cholesky factorisation, 6 triangular solves, 7 refinement
 * residual, 8 LM control, 9 other helpers. */
SC_API uint64_t sc_launch_count(void);
SC_API int32_t sc_profile_begin(void);
SC_API int32_t sc_profile_end(void);
SC_API int32_t sc_profile_read(int32_t kind, int64_t* launches, double* total_ms);

/* Step (a): point-source coherencies of every cluster.
 *   uvw   DEVICE float64 [T][N][3] station coordinates, metres
 *   freqs DEVICE float64 [F] channel frequencies, Hz
 *   sky   clustered sky model (offsets on the HOST, K = d->K clusters)
 *   C     DEVICE out [K][T][B][F] complex (complex64 SC_MIXED, complex128 SC_FP64)
 * SC_FP64 evaluates every (source, baseline, timeslot, channel) phase in
 * float64.  SC_MIXED forms each station's phasor exp(-2 pi i f/c uvw_p.s)
 * from a float64 argument reduced to [-1/2, 1/2) turns, evaluates it in
 * float32 and multiplies station phasors (baseline phase = difference of
 * station phases, exact for point sources), accumulating in float32. */
SC_API int32_t sc_predict_coherencies(const sc_dims* d, const double* uvw,
                                      const double* freqs, const sc_sky* sky,
                                      void* C, int32_t prec, void* ws,
                                      size_t ws_bytes, void* stream);

/* Step (a) for polarised and Gaussian-extended sources: the full 2x2
 * coherency of every cluster,
 *   C_pq(t,f) = sum_s (f/f0)^alpha_s G_s exp(-2 pi i f/c (u l + v m + w (n - 1))) B_s,
 *   B_s = [[I + Q, U + iV], [U - iV, I - Q]]   (unnormalised: an unpolarised
 *         source of flux I gives I * Id, as in sc_predict_coherencies),
 *   G_s = exp(-2 pi^2 (sigma_a^2 u_a^2 + sigma_b^2 u_b^2)),
 * sigma = FWHM / (2 sqrt(2 ln 2)), (u_a, u_b) the baseline (u, v) f/c in
 * wavelengths projected on the major axis (sin pa, cos pa) and the minor
 * axis (cos pa, -sin pa); G_s = 1 when maj = mnr = 0.  The shape is taken on
 * the tangent plane at the source.
 *   uvw, freqs  as sc_predict_coherencies
 *   sky         polarised sky (offsets on the HOST, K = d->K clusters,
 *               at most d->S_max sources per cluster)
 *   C           DEVICE out [K][T][B][F][2][2] complex (complex64 SC_MIXED,
 *               complex128 SC_FP64), the layout of the visibilities
 * SC_MIXED: station phasors as sc_predict_coherencies; the spectral law and
 * the Gaussian's quadratic form are folded per (channel, source) in float64
 * and rounded; float32 attenuation and accumulation.  SC_FP64: everything
 * in float64.  A cluster without sources predicts zeros.
 * Errors: SC_EINVAL (NULL pointers, bad offsets, F * S_max > 2^30),
 * SC_ENOMEM (workspace below sc_workspace_size for d). */
SC_API int32_t sc_predict_coherencies_full(const sc_dims* d, const double* uvw,
                                           const double* freqs, const sc_sky_full* sky,
                                           void* C, int32_t prec, void* ws,
                                           size_t ws_bytes, void* stream);

/* Step (b): residual of one cluster, R = X - J_p (c Id) J_q^H, and its cost
 * sum |R|_F^2.
 *   X     DEVICE [T][B][F][2][2] complex data
 *   C     DEVICE [T][B][F] complex coherencies of the cluster
 *   jones DEVICE complex128 [N][2][2]
 *   R     DEVICE out, same layout as X; may equal X (in place); may be NULL
 *   cost  DEVICE out float64 scalar; may be NULL */
SC_API int32_t sc_residual(const sc_dims* d, const void* X, const void* C,
                           const double* jones, void* R, double* cost,
                           int32_t prec, void* ws, size_t ws_bytes,
                           void* stream);

/* No-allocation variant of sc_residual, for callers that cannot allocate
 * device memory and therefore cannot hand the library a workspace: for
 * example a plug-in inside a host application whose own allocator already
 * owns the whole GPU and offers no way to borrow from it, or a latency-bound
 * loop that forbids cudaMalloc after start-up because an allocation can
 * synchronise the device.  The paper has no counterpart to this call; it
 * exists only for such callers.
 *
 * Same arguments, layouts and results as sc_residual, without the workspace
 * (the cost is summed in a different order, so it agrees to rounding), and
 * the same shape limits (N in [2, 8000], T*F <= 65535).  Its scratch is one
 * 16 MiB array compiled into the library.  Rules:
 *  - the array is device memory taken when the library's device code is
 *    loaded on a GPU and held until the process exits.  Under CUDA's default
 *    lazy module loading that is the first call of this function on the
 *    device (CUDA_MODULE_LOADING=EAGER: context creation).  If your own
 *    allocator will reserve the device, make one call first; otherwise that
 *    first call fails with SC_ECUDA and an out-of-memory message;
 *  - with cost != NULL the problem may have at most 466026 baselines
 *    (N <= 965) in SC_MIXED and 233013 (N <= 683) in SC_FP64; larger ones
 *    are rejected with SC_EINVAL before anything is launched;
 *  - all calls on one device share the array, so calls that overlap on the
 *    GPU (other streams, other host threads) race; serialise them;
 *  - every call made outside stream capture looks up the array's address in
 *    the current CUDA context (cudaGetSymbolAddress), so a driver-API
 *    context of the caller's or a device reset is followed.  A call made
 *    during capture reuses the address found by the last call outside
 *    capture on that device: make one call before capturing, in the context
 *    the graph will run in;
 *  - nothing needs clearing between calls: each call writes all the scratch
 *    it then reads.
 * The error message of this call goes to errbuf (may be NULL), not to
 * sc_last_error(). */
SC_API int32_t sc_residual_noalloc(const sc_dims* d, const void* X, const void* C,
                                   const double* jones, void* R, double* cost,
                                   int32_t prec, void* stream, char* errbuf,
                                   size_t errlen);

/* After calibration: the residual of the whole sky model, optionally
 * corrected for the gains of one direction.  This is the data handed on to
 * imaging once every calibrated cluster has been removed (the abstract
 * states the aim: calibration with minimum artefacts from an incomplete sky
 * model; what remains is the part of the sky the model lacks).
 *   R = V - sum_k J_kp (C_kpq Id) J_kq^H        over all K = d->K clusters
 *   if corr >= 0:  R <- J_cp^{-1} R J_cq^{-H},  c = corr
 * Arguments:
 *   V     DEVICE [T][B][F][2][2] complex observed visibilities
 *   C     DEVICE [K][T][B][F] complex coherencies of every cluster, as
 *         written by sc_predict_coherencies
 *   jones DEVICE complex128 [K][N][2][2], e.g. the output of
 *         sc_calibrate_sage
 *   corr  cluster whose inverse gains are applied, in [0, K); -1 for none
 *   R     DEVICE out, same layout as V; may equal V (in place), must not
 *         otherwise overlap V or C
 *   cost  DEVICE out float64 scalar, sum |R|_F^2 before the correction (the
 *         calibration's total cost); may be NULL
 * Complex types as everywhere: complex64 for SC_MIXED, complex128 for
 * SC_FP64.  In SC_MIXED the Jones are rounded to float32 and the sum is
 * formed in float32; the inverses are formed in float64 and then rounded.
 * A station whose Jones of cluster corr has |det J| <= 1e-12 |J|_F^2 has no
 * usable inverse: the visibilities of all its baselines are set to zero and
 * the device status gets SC_STATUS_SINGULAR (the call still returns SC_OK).
 * Errors: SC_EINVAL (NULL V, C, jones or R; corr outside [-1, K); bad
 * shape), SC_ENOMEM (workspace too small), SC_ECUDA. */
SC_API int32_t sc_residual_all(const sc_dims* d, const void* V, const void* C,
                               const double* jones, int32_t corr, void* R,
                               double* cost, int32_t prec, void* ws,
                               size_t ws_bytes, void* stream);

/* Step (c), the dense solve on its own: factorises a symmetric positive
 * definite matrix as A = L L^T (the factorisation each LM step applies to
 * the damped J^T J) and solves A x = b by the two triangular substitutions.
 *   n     order of A, 1 <= n <= 65536
 *   A     DEVICE in/out, n x n row-major with row pitch lda (>= n) elements,
 *         float (SC_MIXED) / double (SC_FP64); the lower triangle is read.
 *         On return the lower triangle holds L; the strict upper triangle is
 *         unspecified
 *   b     DEVICE float64 [n], may be NULL (then x is not written)
 *   x     DEVICE out float64 [n], may equal b
 *   ws    workspace of at least sc_cholesky_workspace_size() bytes
 *   chol_kernel  SC_CHOL_SIMT or SC_CHOL_TENSOR (SC_MIXED; ignored for SC_FP64)
 * The matrix is copied into the workspace, padded to a multiple of 64 with
 * an identity block, factorised in 64 x 64 tiles and copied back.  A non-positive pivot sets
 * SC_STATUS_NOTPD in the device status (the call returns SC_OK).
 * Errors: SC_EINVAL (n, lda, NULL A, unknown kernel), SC_ENOMEM
 * (workspace), SC_ECUDA. */
SC_API int32_t sc_cholesky_workspace_size(int32_t n, int32_t prec, size_t* bytes);
SC_API int32_t sc_cholesky_solve(int32_t n, void* A, int32_t lda, const double* b, double* x,
                                 int32_t prec, int32_t chol_kernel, void* ws, size_t ws_bytes,
                                 void* stream);

/* Step (c): Gauss-Newton normal equations of one cluster at residual R
 * (= X - model at `jones`):
 *   JhJ   DEVICE out [8N][8N] row-major, float (SC_MIXED) / double (SC_FP64),
 *         the undamped J^T J, both triangles written
 *   Jhr   DEVICE out float64 [8N], J^T r
 * For an unpolarised sky J^T J depends on the data only through
 * w_pq = sum_{t,f} |c_pq(t,f)|^2, which is summed here from C. */
SC_API int32_t sc_lm_normal_eqs(const sc_dims* d, const void* R, const void* C,
                                const double* jones, void* JhJ, double* Jhr,
                                int32_t prec, void* ws, size_t ws_bytes,
                                void* stream);

/* Steps (b)-(c) iterated: Levenberg-Marquardt solve of one cluster against
 * data X, warm-started from and overwriting `jones` (complex128 [N][2][2]).
 *   cost  DEVICE out float64 scalar, final sum |X - model|^2
 *   iters DEVICE out int32 scalar, trial steps taken (<= n_lm)
 * Every iteration stays on the device: the damped J^T J is assembled,
 * factorised by a blocked Cholesky (float32 + float64 refinement for
 * SC_MIXED, float64 for SC_FP64), the step is tried and accepted or rejected
 * by the gain ratio without a host round trip.  A damped matrix that is not
 * positive definite counts as a rejected step (and sets SC_STATUS_NOTPD). */
SC_API int32_t sc_solve_cluster(const sc_dims* d, const void* X, const void* C,
                                double* jones, const sc_lm_opts* opts,
                                double* cost, int32_t* iters, int32_t prec,
                                void* ws, size_t ws_bytes, void* stream);

/* The whole path for one job: predict every cluster, then n_em SAGE sweeps;
 * in each, cluster k = 0..K-1 is solved by LM against
 * X_k = V - sum_{j != k} model_j, kept as a running residual of all
 * clusters plus model_k.
 *   V      DEVICE [T][B][F][2][2] complex observed visibilities
 *   jones  DEVICE complex128 [K][N][2][2], initial guess in, solution out
 *   costs  DEVICE out float64 [K], final LM cost of each cluster in the last
 *          sweep */
SC_API int32_t sc_calibrate_sage(const sc_dims* d, const double* uvw,
                                 const double* freqs, const sc_sky* sky,
                                 const void* V, double* jones,
                                 const sc_sage_opts* opts, double* costs,
                                 int32_t prec, void* ws, size_t ws_bytes,
                                 void* stream);

/* Consecutive time chunks of one observation (one sub-band), calibrated in
 * order with the solver state kept on the device: chunk i runs
 * sc_calibrate_sage on its own data, starting from the solution of chunk
 * i-1 (chunk 0 from `jones`).  Gains drift slowly in time, so each chunk
 * starts near its answer.  Every chunk's solution is written out and is
 * the whole state of the run: calling again with jones = the solution of
 * chunk i and the data of chunks i+1.. continues the run exactly (bit for
 * bit, the kernels being deterministic).
 *   d         shape of ONE chunk (d->T timeslots per chunk)
 *   n_chunks  number of chunks, >= 1
 *   uvw       DEVICE float64 [n_chunks * T][N][3]
 *   freqs     DEVICE float64 [F], the same for every chunk
 *   V         DEVICE [n_chunks][T][B][F][2][2] complex
 *   jones     DEVICE complex128 [K][N][2][2]: initial guess in, solution of
 *             the last chunk out
 *   jones_out DEVICE out complex128 [n_chunks][K][N][2][2], the solution of
 *             every chunk (the checkpoints); may be NULL
 *   costs     DEVICE out float64 [n_chunks][K], final LM cost of each
 *             cluster in the last sweep of each chunk; may be NULL
 * Errors as sc_calibrate_sage; SC_EINVAL also for n_chunks < 1 or
 * n_chunks * T > 65535. */
SC_API int32_t sc_calibrate_chunks(const sc_dims* d, int32_t n_chunks, const double* uvw,
                                   const double* freqs, const sc_sky* sky, const void* V,
                                   double* jones, double* jones_out,
                                   const sc_sage_opts* opts, double* costs, int32_t prec,
                                   void* ws, size_t ws_bytes, void* stream);

/* A whole sc_calibrate_sage call recorded once as a CUDA graph and then
 * replayed.  A job's launch sequence is fixed by its shape and options (the
 * LM and SAGE loops run on the device, with no host decision between
 * kernels), so one capture holds every kernel of the job: a replay costs
 * one graph launch on the host instead of thousands of kernel launches,
 * which is what bounds small jobs (64 stations, one cluster).
 *
 * The graph keeps the pointers, shapes, sky offsets and options given at
 * capture.  To calibrate new data, write it into the same buffers (V, the
 * initial guess in jones, uvw, the sky arrays) before the next replay; a
 * replay then computes exactly what sc_calibrate_sage computes on those
 * contents (bit for bit: same kernels, same order).  Nothing runs during
 * the capture itself.
 *
 * sc_graph_capture_sage: arguments and errors as sc_calibrate_sage, plus
 *   stream  a created stream (not NULL, the legacy default stream, which
 *           cannot be captured), idle on this thread during the call
 *   graph   HOST out: the handle, NULL on error
 * Per-kernel profiling (sc_profile_begin) must be off.  The handle owns
 * host-side driver resources only; it allocates no device memory.
 * sc_graph_launch: replays the graph on `stream` (any stream of the device
 *   it was captured on; NULL = legacy default stream), asynchronously.
 *   Replays that share one workspace must not overlap on the device.
 * sc_graph_destroy: releases the handle (NULL is ignored). */
typedef struct sc_graph sc_graph;
SC_API int32_t sc_graph_capture_sage(const sc_dims* d, const double* uvw,
                                     const double* freqs, const sc_sky* sky,
                                     const void* V, double* jones,
                                     const sc_sage_opts* opts, double* costs,
                                     int32_t prec, void* ws, size_t ws_bytes,
                                     void* stream, sc_graph** graph);
SC_API int32_t sc_graph_launch(sc_graph* graph, void* stream);
SC_API int32_t sc_graph_destroy(sc_graph* graph);

/* Options of the consensus across sub-bands. */
typedef struct sc_consensus_opts {
  sc_sage_opts sage; /* the J-step: SAGE sweeps and LM options of every band */
  int32_t n_admm;    /* consensus iterations (J-step, Z-step, dual step), >= 1 */
  int32_t n_poly;    /* terms of the frequency basis, 1..8, <= n_bands */
  double rho;        /* penalty parameter, >= 0 (0: the bands are independent) */
} sc_consensus_opts;

/* Sub-band calibrations coupled by a smooth frequency model of the Jones.
 * SAGECal calibrates sub-bands in parallel on separate nodes and can tie
 * their solutions together across frequency (paper §1, §2); the paper does
 * not give that algorithm.  This is consensus ADMM in scaled form (Boyd,
 * Parikh, Chu, Peleato & Eckstein 2011, §7.1) on
 *     minimise sum_f f_f(J_f)  subject to  J_f = sum_p basis[f][p] Z_p,
 * f_f the SAGE cost of band f (sum |R|^2 over its data).  Each iteration:
 *   J-step  every band runs sc_calibrate_sage from its current Jones, with
 *           (rho/2) |J_fk - a_fk|_F^2, a_f = basis[f] Z - U_f, added to the
 *           LM cost of each cluster k (as residual rows: J^T J + (rho/2) I,
 *           J^T r + (rho/2)(a - theta)); the first iteration has no
 *           penalty (there is no Z yet), so each band starts alone;
 *   Z-step  Z = (B^T B)^-1 B^T (J + U) per cluster and real parameter;
 *   dual    U_f += J_f - basis[f] Z.
 *   d        shape of ONE band: N, T, F channels per band, K, S_max
 *   n_bands  sub-bands, n_poly..256
 *   uvw      DEVICE float64 [T][N][3], the same for every band
 *   freqs    DEVICE float64 [n_bands][F] channel frequencies of each band
 *   sky      clustered sky model, the same for every band
 *   V        DEVICE [n_bands][T][B][F][2][2] complex data of each band
 *   basis    DEVICE float64 [n_bands][n_poly], e.g. powers of the
 *            normalised band-centre frequency
 *   jones    DEVICE complex128 [n_bands][K][N][2][2], initial guess in,
 *            solution out
 *   dual     DEVICE complex128 [n_bands][K][N][2][2] scaled duals U, in and
 *            out (zero to start; passing the output of a previous call
 *            back continues it)
 *   Z        DEVICE out complex128 [K][n_poly][N][2][2], the frequency model
 *   costs    DEVICE out float64 [n_bands][K], final LM cost of each cluster
 *            in the last iteration, penalty included; may be NULL
 * Workspace: m = ws_bytes / W whole band workspaces, W = sc_workspace_size
 * of d rounded up to 256 bytes (m >= 1).  The J-steps of min(m, n_bands,
 * 16) bands run at once, each band f on internal stream f mod m with band
 * workspace f mod m, joined back to `stream` before each Z-step (events, so
 * a capture of `stream` captures them too); with m = 1 they run one after
 * another on `stream`.  The persistent factorisation of each concurrent
 * band is capped at 2 x SMs / m thread blocks unless lm.max_ctas is set.
 * The result does not depend on m.  The device status at offset 0 of ws
 * gathers every band workspace's status.  Errors as sc_calibrate_sage;
 * SC_EINVAL also for n_bands, n_poly, n_admm or rho out of range.  A
 * singular B^T B raises SC_STATUS_BASIS and zeroes Z. */
SC_API int32_t sc_calibrate_consensus(const sc_dims* d, int32_t n_bands, const double* uvw,
                                      const double* freqs, const sc_sky* sky, const void* V,
                                      const double* basis, double* jones, double* dual, double* Z,
                                      double* costs, const sc_consensus_opts* opts, int32_t prec,
                                      void* ws, size_t ws_bytes, void* stream);

/* One job of a batch: the arguments of sc_calibrate_sage for one sub-band x
 * time chunk, with its own workspace and stream (jobs may differ in every
 * dimension). */
typedef struct sc_job {
  sc_dims dims;
  const double* uvw;
  const double* freqs;
  sc_sky sky;
  const void* V;
  double* jones;
  double* costs;
  void* ws;
  size_t ws_bytes;
  void* stream;
} sc_job;

/* Many independent calibrations at once (paper §1: SAGECal distributes
 * frequency bands; here sub-bands and time chunks of uneven size share one
 * GPU).  Each job is calibrated exactly as by sc_calibrate_sage on its own
 * stream with its own workspace; a pool of host threads enqueues them so
 * that they overlap on the device, and the factorisation kernel of each job
 * is capped (opts->lm.max_ctas, or an even share of the GPU when 0).  Results
 * of a job do not depend on the other jobs.  Returns when every job has been
 * enqueued; the first error (if any) is returned and later jobs are still
 * attempted.  The device takes the streams' launches through a fixed number
 * of hardware work queues (CUDA_DEVICE_MAX_CONNECTIONS, 8 unless set before
 * the process creates its CUDA context, at most 32); streams that share a
 * queue wait on each other's launches, so overlap needs it raised (the
 * Python package sets 32 at import unless the variable is set). */
SC_API int32_t sc_calibrate_batch(const sc_job* jobs, int32_t n_jobs,
                                  const sc_sage_opts* opts, int32_t prec);

/* Workspace of sc_calibrate_batched for these jobs (dims[n_jobs]; every job
 * the N and K of job 0): one block per job holding the buffers of its
 * cluster solves (Jones and LM state, statistics, the 8N x 8N matrix and
 * its factor), about 4 (8 N)^2 bytes per job in SC_MIXED, and the task
 * order of the batched factorisation (4 bytes per factorisation task of
 * every job).  SC_EINVAL if the dimensions are invalid or differ in N or K. */
SC_API int32_t sc_batched_workspace_size(const sc_dims* dims, int32_t n_jobs, int32_t prec, size_t* bytes);

/* Many calibrations of equal station count N and cluster count K in lock
 * step (paper §1: sub-bands and time chunks calibrated side by side; the
 * jobs may differ in T, F, S_max, sky and data).  Each job is calibrated
 * exactly as by sc_calibrate_sage with its own workspace (jobs[g].ws: its
 * coherencies and running residual): the result of every job is bit for bit
 * the one sc_calibrate_sage gives it.  Per cluster, each job's statistics
 * pass runs over its own data; then every stage of the LM loop (Alg. 3.16
 * of Madsen, Nielsen & Tingleff: assembly, factorisation, solves,
 * refinement, trial, evaluation, decision) is one launch over all jobs.
 * The factorisations of all jobs are one persistent kernel taking the
 * tasks of the jobs' tile lists merged into one list in which each job
 * keeps its own order.  window 0 interleaves the lists (task t of job g at
 * position t * n_jobs + g: every job advances together, and the blocks
 * waiting on one job's dependency chain are few among those working on the
 * others).  window W in [1, 2^20] staggers the jobs instead: job g starts
 * its list when job g - W is about to finish, so that about W matrices are
 * read at a time; sc_tune_batched measures the choices.  ws:
 * sc_batched_workspace_size bytes, 256-byte aligned, device memory owned by
 * the caller.  Everything runs on `stream`, after what is already queued on
 * each job's stream, and each job's stream then waits for the batch
 * (events).  opts->lm.max_ctas caps the factorisation's blocks (0: all
 * resident ones); opts->lm.chol_kernel must be SC_CHOL_SIMT.  Errors as
 * sc_calibrate_sage (SC_EINVAL also for a window outside [0, 2^20]); a job's device status
 * word gathers its solves'. */
SC_API int32_t sc_calibrate_batched(const sc_job* jobs, int32_t n_jobs, const sc_sage_opts* opts, int32_t prec,
                                    int32_t window, void* ws, size_t ws_bytes, void* stream);

/* Autotuner of the batched factorisation: for each of windows[n_windows]
 * (each in [1, 2^20]; one above (n_jobs - 1) x the tasks of one job
 * orders the tasks as the interleave does), times `reps` factorisations of the
 * jobs' matrix order (identity matrices: the arithmetic takes the same time
 * on any values) in the batch workspace ws (sc_batched_workspace_size of
 * dims), after one untimed run, with CUDA events on `stream`; writes the
 * mean milliseconds per factorisation to ms_out[n_windows] and the fastest
 * window to *best.  Synchronises `stream` (the one call of this library
 * that does); overwrites ws.  SC_EINVAL for bad arguments or a batch too
 * large for a staggered order. */
SC_API int32_t sc_tune_batched(const sc_dims* dims, int32_t n_jobs, int32_t prec, const int32_t* windows,
                               int32_t n_windows, int32_t reps, double* ms_out, int32_t* best, void* ws,
                               size_t ws_bytes, void* stream);

/* Host only, for tests: position in the merged factorisation task list of
 * task t of job g, out[g * n + t], n the tasks per job of nT tile rows, for
 * n_jobs jobs staggered over `window` jobs (as sc_calibrate_batched orders
 * them).  cap: entries of out (>= n_jobs * n). */
SC_API int32_t sc_batch_order(int32_t nT, int32_t n_jobs, int32_t window, int32_t* out, int64_t cap);

#ifdef __cplusplus
}
#endif

#endif /* SAGECAL_GB_H */
