// Steps (b) and (c, gradient half) inside the LM loop, from per-baseline
// statistics of the data.
//
// Within one cluster's solve the data X and the coherencies c are fixed (X is
// the E-step data Xin + c G_old of SAGE, or the caller's data), and one Jones
// set spans all T and F.  With G = J_p J_q^H the residual of visibility
// (t, f) of baseline pq is r = X - c G, so over t and f
//     cost_pq = S - 2 Re <G, rhoX> + W |G|_F^2,      rho_pq = sum conj(c) r = rhoX - W G,
//     S = sum |X|_F^2,   rhoX = sum conj(c) X,   W = sum |c|^2,
// with <A, B> = sum_ij conj(A_ij) B_ij.  k_lm_stats forms (S, rhoX, W) once
// per solve, one pass over X and C; every LM evaluation then reads those ten
// numbers per baseline instead of the visibilities (k_lm_eval).  The
// gradient of the cost with respect to J_p is -2 rho_pq J_q and with respect
// to J_q -2 rho_pq^H J_p, so J^T r of station s is sum_o rho J_o (s = p) or
// rho^H J_o (s = q); the diagonal block of J^T J of station s is the real
// form of dJ_s -> dJ_s H_s, H_s = sum_o W_so J_o^H J_o (normal_eqs.cu).
//
// At a good fit the three terms of the cost nearly cancel, so the statistics
// of float32 data are kept to about twice float32's precision, as unevaluated
// pairs hi + lo of floats: every product is split exactly (TwoProduct by
// FMA) and the sums are compensated (TwoSum; the Sum2 algorithm of Ogita,
// Rump & Oishi 2005), and the expansion is evaluated in the same pair
// arithmetic.  The cost is then that of the float32 data to about 1e-12 of
// S, with no float64 arithmetic (float64 is slow on this GPU).  The float64
// path keeps everything in float64.
#include <algorithm>

#include "sc_common.cuh"

namespace sc {

constexpr int kStatV = 10;  // S, rhoX (8), W
constexpr int kStatThreads = 256;
// Blocks of the float32 pass: 128 threads.  At its 72 registers a thread,
// an SM holds 7 such blocks (28 warps) against 3 of 256 threads (24 warps);
// each item's sums stay in one thread, so the block size does not change
// them.
constexpr int kStat32Threads = 128;

// ---- pairs of floats -------------------------------------------------------------------------
//
// The _rn intrinsics are never fused into an FMA, which the error terms need.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF two_sum(float a, float b) {  // a + b = s + e exactly
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
__device__ __forceinline__ FF two_prod(float a, float b) {  // a b = p + e exactly
  const float p = __fmul_rn(a, b);
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF fast_renorm(float s, float e) {  // |s| >= |e|
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
// a + b; absolute error about 2^-44 (|a| + |b|)
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  const FF s = two_sum(a.hi, b.hi);
  return fast_renorm(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ FF ff_mul_f(FF a, float b) {
  const FF p = two_prod(a.hi, b);
  return fast_renorm(p.hi, fmaf(a.lo, b, p.lo));
}
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const FF p = two_prod(a.hi, b.hi);
  return fast_renorm(p.hi, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, p.lo)));
}
// s += a b, as in Sum2: the error terms gather in s.lo, renormalised once at
// the end
__device__ __forceinline__ void ff_acc_prod(FF& s, float a, float b) {
  const FF p = two_prod(a, b);
  const FF t = two_sum(s.hi, p.hi);
  s.hi = t.hi;
  s.lo = __fadd_rn(s.lo, __fadd_rn(t.lo, p.lo));
}

// ---- the same on pairs of sums at once -------------------------------------------------------
//
// Blackwell's packed float32 instructions (add / sub / mul / fma .rn.f32x2)
// round each lane exactly as the scalar instruction does, so two
// accumulators advance in one instruction with the arithmetic above.
__device__ __forceinline__ unsigned long long pk2(float2 a) { return *reinterpret_cast<unsigned long long*>(&a); }
__device__ __forceinline__ float2 upk2(unsigned long long d) { return *reinterpret_cast<float2*>(&d); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {  // a b + c, rounded once
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
struct FF2 {  // two pairs: lane x and lane y
  float2 hi, lo;
};
// s += a b per lane, as ff_acc_prod
__device__ __forceinline__ void ff2_acc_prod(FF2& s, float2 a, float2 b) {
  const float2 p = mul2(a, b);
  const float2 e = fma2(a, b, make_float2(-p.x, -p.y));
  const float2 t = add2(s.hi, p);
  const float2 z = sub2(t, s.hi);
  const float2 tl = add2(sub2(s.hi, sub2(t, z)), sub2(p, z));
  s.hi = t;
  s.lo = add2(s.lo, add2(tl, e));
}

// The ten sums of one (chunk, baseline) item in float32 pairs: rhoX as its
// (re, im) pairs, two sums per packed instruction, each lane with the
// operations (and order) of the scalar sum; S and W stay scalar sums in
// their order (squares of re, im of each entry in turn; c.re^2, c.im^2),
// so the statistics are the bits the scalar version gives.
struct Stat32 {
  FF S, W;
  FF2 rho[4];
};
__device__ __forceinline__ void stat_zero(Stat32& a) {
  const FF2 z = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  a.S = {0.f, 0.f};
  a.W = {0.f, 0.f};
#pragma unroll
  for (int e = 0; e < 4; ++e) a.rho[e] = z;
}
__device__ __forceinline__ void stat_add(Stat32& a, const m22<float>& x, cx<float> c) {
  const float2 xs[4] = {make_float2(x.a.re, x.a.im), make_float2(x.b.re, x.b.im), make_float2(x.c.re, x.c.im),
                        make_float2(x.d.re, x.d.im)};
  const float2 cr = make_float2(c.re, c.re), ci = make_float2(c.im, -c.im);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    ff_acc_prod(a.S, xs[e].x, xs[e].x);
    ff_acc_prod(a.S, xs[e].y, xs[e].y);
    // conj(c) x = (c.re x.re + c.im x.im, c.re x.im - c.im x.re)
    ff2_acc_prod(a.rho[e], cr, xs[e]);
    ff2_acc_prod(a.rho[e], ci, make_float2(xs[e].y, xs[e].x));
  }
  ff_acc_prod(a.W, c.re, c.re);
  ff_acc_prod(a.W, c.im, c.im);
}

// The ten sums of one (chunk, baseline) item in float64.
__device__ __forceinline__ void stat_add(double (&a)[kStatV], const m22<double>& x, cx<double> c) {
  const double xs[8] = {x.a.re, x.a.im, x.b.re, x.b.im, x.c.re, x.c.im, x.d.re, x.d.im};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const double xr = xs[2 * e], xi = xs[2 * e + 1];
    a[0] = fma(xr, xr, fma(xi, xi, a[0]));
    a[1 + 2 * e] = fma(c.re, xr, fma(c.im, xi, a[1 + 2 * e]));
    a[2 + 2 * e] = fma(c.re, xi, fma(-c.im, xr, a[2 + 2 * e]));
  }
  a[9] = fma(c.re, c.re, fma(c.im, c.im, a[9]));
}

// Layout of the statistics: [chunk][value][B] doubles in float64; in float32
// [chunk][value][hi, lo][B] floats (the same bytes).
__device__ __forceinline__ void stat_store(double* stat, int64_t B, int chunk, int64_t b, const double (&a)[kStatV]) {
  double* o = stat + (size_t)chunk * kStatV * B + b;
#pragma unroll
  for (int i = 0; i < kStatV; ++i) o[(size_t)i * B] = a[i];
}
__device__ __forceinline__ void stat_store(double* stat, int64_t B, int chunk, int64_t b, const FF (&a)[kStatV]) {
  float* o = reinterpret_cast<float*>(stat) + (size_t)chunk * 2 * kStatV * B + b;
#pragma unroll
  for (int i = 0; i < kStatV; ++i) {
    const FF r = fast_renorm(a[i].hi, a[i].lo);
    o[(size_t)(2 * i) * B] = r.hi;
    o[(size_t)(2 * i + 1) * B] = r.lo;
  }
}
__device__ __forceinline__ void stat_store(double* stat, int64_t B, int chunk, int64_t b, const Stat32& a) {
  FF v[kStatV];
  v[0] = a.S;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    v[1 + 2 * e] = {a.rho[e].hi.x, a.rho[e].lo.x};
    v[2 + 2 * e] = {a.rho[e].hi.y, a.rho[e].lo.y};
  }
  v[9] = a.W;
  stat_store(stat, B, chunk, b, v);
}

// ---- the statistics pass ---------------------------------------------------------------------
//
// One thread per (timeslot chunk, baseline) item, grid-stride; X = Xin + c G_old
// when FL has P_OLD (formed in R, as the visibility pass forms it), else
// X = Xin.
//
// float64: a plain loop.  float32: the pair arithmetic costs about 260
// instructions per visibility, too little work per load for the warps of an
// SM to hide DRAM latency, so every thread streams its own sequence of
// visibilities through a ring of kRing stages in shared memory filled by
// cp.async, the prefetch cursor kRing - 1 visibilities ahead of the
// arithmetic and crossing item boundaries.  A thread reads only the slots it
// filled, so cp.async.wait_group alone orders the data.  Slots are laid out
// [stage][part][thread], conflict-free for a warp's 16- and 8-byte reads.
template <int FL>
__global__ void __launch_bounds__(kStatThreads) k_lm_stats64(int N, int T, int F, int64_t B, int nchunk, int tchunk,
                                                           const double* __restrict__ Xin,
                                                           const double* __restrict__ C,
                                                           const double* __restrict__ J_old, double* __restrict__ stat,
                                                           int* __restrict__ nchunk_out) {
  if (nchunk_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *nchunk_out = nchunk;
  const int64_t n_items = (int64_t)nchunk * B;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_items;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int chunk = (int)(idx / B);
    const int64_t b = idx - (int64_t)chunk * B;
    m22<double> Go = mzero<double>();
    if (FL & P_OLD) {
      int p, q;
      bl_pair(b, N, p, q);
      Go = mul_h(load_jones<double>(J_old, p), load_jones<double>(J_old, q));
    }
    double a[kStatV];
#pragma unroll
    for (int i = 0; i < kStatV; ++i) a[i] = 0.0;
    const int t0 = chunk * tchunk, t1 = min(T, t0 + tchunk);
    for (int t = t0; t < t1; ++t) {
      const size_t v0 = ((size_t)t * B + b) * F;
      for (int f = 0; f < F; ++f) {
        const size_t v = v0 + f;
        m22<double> x = ld_vis(Xin + 8 * v);
        const cx<double> c = ld_c(C + 2 * v);
        if (FL & P_OLD) x = x + smul(c, Go);
        stat_add(a, x, c);
      }
    }
    stat_store(stat, B, chunk, b, a);
  }
}

namespace {
__device__ __forceinline__ void st_cp8(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void st_cp16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void st_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int W>
__device__ __forceinline__ void st_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(W) : "memory"); }
}  // namespace

constexpr int kRing = 4;
constexpr size_t kRingSmem = (size_t)kRing * kStat32Threads * (2 * 16 + 8);

// Position in one thread's sequence: item idx = (chunk, b), timeslot t of
// [t0, t1), channel f.
struct StatCursor {
  int64_t idx, b;
  int chunk, t, t1, f;
  __device__ void start(int64_t i, int64_t B, int T, int tchunk) {
    idx = i;
    chunk = (int)(i / B);
    b = i - (int64_t)chunk * B;
    t = chunk * tchunk;
    t1 = min(T, t + tchunk);
    f = 0;
  }
  // advances one visibility; true when the item ended
  __device__ bool next(int F) {
    if (++f < F) return false;
    f = 0;
    return ++t == t1;
  }
};

template <int FL>
__global__ void __launch_bounds__(kStat32Threads) k_lm_stats32(int N, int T, int F, int64_t B, int nchunk, int tchunk,
                                                           const float* __restrict__ Xin,
                                                           const float* __restrict__ C,
                                                           const double* __restrict__ J_old, double* __restrict__ stat,
                                                           int* __restrict__ nchunk_out) {
  if (nchunk_out != nullptr && blockIdx.x == 0 && threadIdx.x == 0) *nchunk_out = nchunk;
  extern __shared__ __align__(16) unsigned char st_smem[];
  float4* xring = reinterpret_cast<float4*>(st_smem);                                        // [kRing][2][T]
  float2* cring = reinterpret_cast<float2*>(st_smem + (size_t)kRing * 2 * kStat32Threads * 16);  // [kRing][T]
  const int tid = threadIdx.x;
  const int64_t n_items = (int64_t)nchunk * B;
  const int64_t stride = (int64_t)gridDim.x * kStat32Threads;
  const int64_t first = (int64_t)blockIdx.x * kStat32Threads + tid;
  StatCursor pf, cs;  // prefetch and consume cursors
  if (first < n_items) pf.start(first, B, T, tchunk);
  else pf.idx = n_items;
  cs = pf;
  int pf_stage = 0, cs_stage = 0;
  auto issue = [&]() {
    if (pf.idx < n_items) {
      const size_t v = ((size_t)pf.t * B + pf.b) * F + pf.f;
      st_cp16(&xring[(pf_stage * 2) * kStat32Threads + tid], Xin + 8 * v);
      st_cp16(&xring[(pf_stage * 2 + 1) * kStat32Threads + tid], Xin + 8 * v + 4);
      st_cp8(&cring[pf_stage * kStat32Threads + tid], C + 2 * v);
      if (pf.next(F)) {
        const int64_t n = pf.idx + stride;
        if (n < n_items) pf.start(n, B, T, tchunk);
        else pf.idx = n_items;
      }
    }
    st_commit();
    pf_stage = pf_stage + 1 == kRing ? 0 : pf_stage + 1;
  };
#pragma unroll
  for (int k = 0; k < kRing - 1; ++k) issue();
  m22<float> Go = mzero<float>();
  auto item_begin = [&]() {
    if ((FL & P_OLD) && cs.idx < n_items) {
      int p, q;
      bl_pair(cs.b, N, p, q);
      Go = mul_h(load_jones<float>(J_old, p), load_jones<float>(J_old, q));
    }
  };
  item_begin();
  Stat32 a;
  stat_zero(a);
  while (cs.idx < n_items) {
    issue();
    st_wait<kRing - 1>();  // the consume stage has landed
    const float4 u = xring[(cs_stage * 2) * kStat32Threads + tid];
    const float4 w = xring[(cs_stage * 2 + 1) * kStat32Threads + tid];
    const float2 cc = cring[cs_stage * kStat32Threads + tid];
    cs_stage = cs_stage + 1 == kRing ? 0 : cs_stage + 1;
    m22<float> x = {{u.x, u.y}, {u.z, u.w}, {w.x, w.y}, {w.z, w.w}};
    const cx<float> c = {cc.x, cc.y};
    if (FL & P_OLD) x = x + smul(c, Go);
    stat_add(a, x, c);
    if (cs.next(F)) {
      stat_store(stat, B, cs.chunk, cs.b, a);
      stat_zero(a);
      const int64_t n = cs.idx + stride;
      if (n < n_items) cs.start(n, B, T, tchunk);
      else cs.idx = n_items;
      item_begin();
    }
  }
  st_wait<0>();
}

// Most timeslot chunks of the statistics pass: 16, fewer when the baselines
// alone give four items per thread a GPU of kMaxSMs multiprocessors holds.
static int stats_max_chunks(int T, int64_t B) {
  const int64_t by_size = (int64_t)kMaxSMs * 2048 * 4 / std::max<int64_t>(B, 1);
  return (int)std::max<int64_t>(1, std::min<int64_t>(std::min(T, 16), by_size));
}

// Timeslot chunks of the statistics pass: as few as give at least half as
// many (chunk, baseline) items as there are resident threads.  Every LM
// evaluation reads and adds the statistics of every chunk, so a chunk more
// costs each evaluation 80 bytes per baseline; the pass itself keeps its
// loads in flight through the ring, not through the number of threads.
static void stats_chunks(int T, int64_t B, int64_t slots, int* nchunk, int* tchunk) {
  const int64_t want = (slots / 2 + std::max<int64_t>(B, 1) - 1) / std::max<int64_t>(B, 1);
  const int n = (int)std::max<int64_t>(1, std::min<int64_t>(want, stats_max_chunks(T, B)));
  *tchunk = (T + n - 1) / n;
  *nchunk = (T + *tchunk - 1) / *tchunk;
}

size_t lm_stats_doubles(int T, int64_t B) { return (size_t)stats_max_chunks(T, B) * kStatV * (size_t)B; }

template <typename R>
struct StatsKernel;
template <>
struct StatsKernel<float> {
  template <int FL>
  static const void* fn() { return reinterpret_cast<const void*>(&k_lm_stats32<FL>); }
  static constexpr size_t smem = kRingSmem;
  static constexpr int threads = kStat32Threads;
};
template <>
struct StatsKernel<double> {
  template <int FL>
  static const void* fn() { return reinterpret_cast<const void*>(&k_lm_stats64<FL>); }
  static constexpr size_t smem = 0;
  static constexpr int threads = kStatThreads;
};

template <typename R, int FL>
static cudaError_t go_stats(const Shape& s, const R* Xin, const R* C, const double* J_old, double* stat,
                            int* nchunk, int* nchunk_dev, cudaStream_t st) {
  using K = StatsKernel<R>;
  // resident blocks of this instantiation, computed once (thread-safe static)
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* f = K::template fn<FL>();
    if (K::smem > 48 * 1024) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)K::smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, K::threads, K::smem);
    return std::max(1, std::min(sms, kMaxSMs) * std::max(per, 1));
  }();
  int nc = 0, tc = 0;
  stats_chunks(s.T, s.B, (int64_t)resident * K::threads, &nc, &tc);
  *nchunk = nc;
  const int64_t items = (int64_t)nc * s.B;
  const unsigned grid = (unsigned)std::min<int64_t>((items + K::threads - 1) / K::threads, resident);
  if constexpr (sizeof(R) == 4)
    k_lm_stats32<FL><<<grid, K::threads, K::smem, st>>>(s.N, s.T, s.F, s.B, nc, tc, Xin, C, J_old, stat,
                                                          nchunk_dev);
  else
    k_lm_stats64<FL><<<grid, kStatThreads, 0, st>>>(s.N, s.T, s.F, s.B, nc, tc, Xin, C, J_old, stat, nchunk_dev);
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_lm_stats(const Shape& s, const R* Xin, const R* C, const double* J_old, double* stat,
                            int* nchunk, cudaStream_t st, int* nchunk_dev) {
  return J_old != nullptr ? go_stats<R, P_OLD>(s, Xin, C, J_old, stat, nchunk, nchunk_dev, st)
                          : go_stats<R, 0>(s, Xin, C, J_old, stat, nchunk, nchunk_dev, st);
}
template cudaError_t launch_lm_stats<float>(const Shape&, const float*, const float*, const double*, double*, int*,
                                            cudaStream_t, int*);
template cudaError_t launch_lm_stats<double>(const Shape&, const double*, const double*, const double*, double*,
                                             int*, cudaStream_t, int*);

// ---- one LM evaluation: per-station sums from the statistics ------------------------------
//
// Stations are cut into tiles of kST; a block takes one pair of station tiles
// (Pt <= Qt), one thread per baseline (p, q), p in tile Pt, q in tile Qt,
// p < q.  A thread forms from its baseline's statistics, in float64, the
// cost and rho at J, then (in R) what the baseline adds to station p
// (rho J_q, W J_q^H J_q) and to station q (rho^H J_p, W J_p^H J_p).  The
// block sums the p parts over the kST baselines of a tile row (shuffles
// within a half-warp) and the q parts over the kST baselines of a tile
// column (shared memory), and writes one partial per tile row and column.
// k_station_sum adds, for each station, the partials of the tiles of its
// tile row and column in a fixed order, so the sums are deterministic.
constexpr int kST = 16;
constexpr int kRowV = 13;                           // J^T r (8), H (4), cost
constexpr int kColV = 12;                           // J^T r (8), H (4)
constexpr int kPartStride = kST * (kRowV + kColV);  // doubles per tile pair

__host__ __device__ __forceinline__ int tile_pair(int Pt, int Qt, int nS) {
  return Pt * nS - Pt * (Pt - 1) / 2 + (Qt - Pt);
}

size_t lm_part_doubles(int N) {
  const int nS = (N + kST - 1) / kST;
  return (size_t)nS * (nS + 1) / 2 * kPartStride;
}

// The baseline's cost and rho at J from its statistics (summed over the
// chunks).  float32 statistics: pair arithmetic with G = J_p J_q^H formed in
// float32 (the model the visibility pass would form), so the three terms of
// the cost are those of one and the same G; rho is returned rounded.
__device__ __forceinline__ void eval_baseline(const double* stat, int64_t B, int nchunk, int64_t b, bool sub,
                                              const m22<float>& Jp, const m22<float>& Jq, FF& cost,
                                              m22<float>& rho, float& W) {
  const float* st = reinterpret_cast<const float*>(stat);
  FF v[kStatV];
#pragma unroll
  for (int i = 0; i < kStatV; ++i) v[i] = {0.f, 0.f};
  for (int c = 0; c < nchunk; ++c) {
    const float* src = st + (size_t)c * 2 * kStatV * B + b;
#pragma unroll
    for (int i = 0; i < kStatV; ++i) v[i] = ff_add(v[i], FF{src[(size_t)(2 * i) * B], src[(size_t)(2 * i + 1) * B]});
  }
  W = v[9].hi;
  if (!sub) {
    cost = v[0];
    rho = {{v[1].hi, v[2].hi}, {v[3].hi, v[4].hi}, {v[5].hi, v[6].hi}, {v[7].hi, v[8].hi}};
    return;
  }
  const m22<float> G = mul_h(Jp, Jq);
  const float g[8] = {G.a.re, G.a.im, G.b.re, G.b.im, G.c.re, G.c.im, G.d.re, G.d.im};
  // cost = S - 2 Re <G, rhoX> + W |G|^2,  rho = rhoX - W G
  FF cross = {0.f, 0.f}, g2 = {0.f, 0.f};
  float r[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    cross = ff_add(cross, ff_mul_f(v[1 + k], g[k]));
    g2 = ff_add(g2, two_prod(g[k], g[k]));
    const FF rk = ff_add(v[1 + k], ff_mul_f(v[9], -g[k]));
    r[k] = __fadd_rn(rk.hi, rk.lo);
  }
  cost = ff_add(ff_add(v[0], ff_mul_f(cross, -2.f)), ff_mul(v[9], g2));
  rho = {{r[0], r[1]}, {r[2], r[3]}, {r[4], r[5]}, {r[6], r[7]}};
}
__device__ __forceinline__ void eval_baseline(const double* stat, int64_t B, int nchunk, int64_t b, bool sub,
                                              const m22<double>& Jp, const m22<double>& Jq, double& cost,
                                              m22<double>& rho, double& W) {
  double v[kStatV];
#pragma unroll
  for (int i = 0; i < kStatV; ++i) v[i] = 0.0;
  for (int c = 0; c < nchunk; ++c) {
    const double* src = stat + (size_t)c * kStatV * B + b;
#pragma unroll
    for (int i = 0; i < kStatV; ++i) v[i] += src[(size_t)i * B];
  }
  const m22<double> rX = {{v[1], v[2]}, {v[3], v[4]}, {v[5], v[6]}, {v[7], v[8]}};
  W = v[9];
  cost = v[0];
  rho = rX;
  if (!sub) return;
  const m22<double> G = mul_h(Jp, Jq);
  const double cross = G.a.re * rX.a.re + G.a.im * rX.a.im + G.b.re * rX.b.re + G.b.im * rX.b.im +
                       G.c.re * rX.c.re + G.c.im * rX.c.im + G.d.re * rX.d.re + G.d.im * rX.d.im;
  cost = v[0] - 2.0 * cross + W * frob2(G);
  rho = rX - smul(cmk(W, 0.0), G);
}

// the cost of a tile row, summed over the kST lanes of a half-warp; returned
// in float64 by every lane
__device__ __forceinline__ double row_cost_sum(FF c) {
#pragma unroll
  for (int o = kST / 2; o > 0; o >>= 1) {
    const FF d = {__shfl_xor_sync(0xffffffffu, c.hi, o), __shfl_xor_sync(0xffffffffu, c.lo, o)};
    c = ff_add(c, d);
  }
  return (double)c.hi + (double)c.lo;
}
__device__ __forceinline__ double row_cost_sum(double c) {
#pragma unroll
  for (int o = kST / 2; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  return c;
}

template <typename R> struct CostT;
template <> struct CostT<float> { using T = FF; __device__ static FF zero() { return {0.f, 0.f}; } };
template <> struct CostT<double> { using T = double; __device__ static double zero() { return 0.0; } };

template <typename R, bool SUB>
__global__ void __launch_bounds__(kST * kST) k_lm_eval(int N, int64_t B, int nS, int nchunk,
                                                     const double* __restrict__ stat,
                                                     const double* __restrict__ J, double* __restrict__ part,
                                                     const LMState* __restrict__ lm, size_t js,
                                                     const int* __restrict__ nchunk_dev) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm != nullptr && (lm->done | lm->skip)) return;
  stat = job_ptr(stat, js, job);
  J = job_ptr(J, js, job);
  part = job_ptr(part, js, job);
  if (nchunk_dev != nullptr) nchunk = *job_ptr(nchunk_dev, js, job);
  __shared__ R colbuf[kColV][kST][kST + 1];
  const int pair = blockIdx.x;
  // tile pairs (Pt, Qt), Pt <= Qt, are numbered like the baselines of nS + 1
  // stations: pair = bl_index(Pt, Qt + 1, nS + 1)
  int Pt, q1;
  bl_pair(pair, nS + 1, Pt, q1);
  const int Qt = q1 - 1;
  const int pl = threadIdx.x / kST, ql = threadIdx.x % kST;
  const int p = kST * Pt + pl, q = kST * Qt + ql;
  const bool act = p < q && q < N;
  typename CostT<R>::T cost = CostT<R>::zero();
  R w = 0;
  m22<R> rh = mzero<R>(), Jp = mzero<R>(), Jq = mzero<R>();
  if (act) {
    Jp = load_jones<R>(J, p);
    Jq = load_jones<R>(J, q);
    eval_baseline(stat, B, nchunk, bl_index(p, q, N), SUB, Jp, Jq, cost, rh, w);
  }
  double* out = part + (size_t)pair * kPartStride;
  // station p's part, summed over the tile row: the kST lanes of a half-warp
  // hold the baselines (p, q) of one p
  {
    R rv[kRowV - 1];
    const m22<R> gp = mul(rh, Jq);
    const cx<R> h = cmulc(Jq.a, Jq.b) + cmulc(Jq.c, Jq.d);
    rv[0] = gp.a.re, rv[1] = gp.a.im, rv[2] = gp.b.re, rv[3] = gp.b.im;
    rv[4] = gp.c.re, rv[5] = gp.c.im, rv[6] = gp.d.re, rv[7] = gp.d.im;
    rv[8] = w * (norm2(Jq.a) + norm2(Jq.c));
    rv[9] = w * (norm2(Jq.b) + norm2(Jq.d));
    rv[10] = w * h.re, rv[11] = w * h.im;
#pragma unroll
    for (int v = 0; v < kRowV - 1; ++v) {
#pragma unroll
      for (int o = kST / 2; o > 0; o >>= 1) rv[v] += __shfl_xor_sync(0xffffffffu, rv[v], o);
    }
    const double csum = row_cost_sum(cost);
#pragma unroll
    for (int v = 0; v < kRowV - 1; ++v)
      if (ql == v) out[pl * kRowV + v] = (double)rv[v];
    if (ql == kRowV - 1) out[pl * kRowV + kRowV - 1] = csum;
  }
  // station q's part, summed over the tile column through shared memory
  {
    const m22<R> gq = mul(hconj(rh), Jp);
    const cx<R> h = cmulc(Jp.a, Jp.b) + cmulc(Jp.c, Jp.d);
    colbuf[0][pl][ql] = gq.a.re, colbuf[1][pl][ql] = gq.a.im;
    colbuf[2][pl][ql] = gq.b.re, colbuf[3][pl][ql] = gq.b.im;
    colbuf[4][pl][ql] = gq.c.re, colbuf[5][pl][ql] = gq.c.im;
    colbuf[6][pl][ql] = gq.d.re, colbuf[7][pl][ql] = gq.d.im;
    colbuf[8][pl][ql] = w * (norm2(Jp.a) + norm2(Jp.c));
    colbuf[9][pl][ql] = w * (norm2(Jp.b) + norm2(Jp.d));
    colbuf[10][pl][ql] = w * h.re;
    colbuf[11][pl][ql] = w * h.im;
  }
  __syncthreads();
  if (threadIdx.x < kST * kColV) {
    const int v = threadIdx.x / kST, c = threadIdx.x % kST;
    R t = 0;
#pragma unroll
    for (int r = 0; r < kST; ++r) t += colbuf[v][r][c];
    out[kST * kRowV + c * kColV + v] = (double)t;
  }
}

template <typename R>
cudaError_t launch_lm_eval(const Shape& s, bool sub, const double* stat, int nchunk, const double* J, double* part,
                           const LMState* lm, cudaStream_t st, const Batch& bt, const int* nchunk_dev) {
  const int nS = (s.N + kST - 1) / kST, pairs = nS * (nS + 1) / 2;
  const dim3 grd(pairs, 1, bt.G);
  if (sub) k_lm_eval<R, true><<<grd, kST * kST, 0, st>>>(s.N, s.B, nS, nchunk, stat, J, part, lm, bt.js, nchunk_dev);
  else k_lm_eval<R, false><<<grd, kST * kST, 0, st>>>(s.N, s.B, nS, nchunk, stat, J, part, lm, bt.js, nchunk_dev);
  return cudaGetLastError();
}
template cudaError_t launch_lm_eval<float>(const Shape&, bool, const double*, int, const double*, double*,
                                           const LMState*, cudaStream_t, const Batch&, const int*);
template cudaError_t launch_lm_eval<double>(const Shape&, bool, const double*, int, const double*, double*,
                                            const LMState*, cudaStream_t, const Batch&, const int*);

// One warp per station s.  Lane (h, v), h = lane / 16 and v = lane % 16 < 13,
// adds value v of every other partial of the list
//   the row partials of tiles (St, Qt), Qt = St..nS-1,
//   then the column partials of tiles (Pt, St), Pt = 0..St,
// starting at partial h; one shuffle then joins the two halves (a fixed
// order).  The quadratic penalty of the consensus step,
// pen_w |theta_s - a_s|^2, enters here as residual rows
// sqrt(pen_w) (a - theta): J^T r += pen_w (a - theta), the real diagonal of H
// (hence of J^T J) += pen_w, cost += pen_w |theta - a|^2.
constexpr int kSumThreads = 64;  // two stations per block: the float64 adds spread over every SM
__global__ void __launch_bounds__(kSumThreads) k_station_sum(int N, int nS, const double* __restrict__ part,
                                                             const double* __restrict__ J, double* __restrict__ g,
                                                             double* __restrict__ H, double* __restrict__ cpart,
                                                             double* __restrict__ gmax,
                                                             const LMState* __restrict__ lm,
                                                             const double* __restrict__ pen, double pen_w,
                                                             size_t js) {
  const int job = blockIdx.z;
  lm = job_ptr(lm, js, job);
  if (lm != nullptr && (lm->done | lm->skip)) return;
  part = job_ptr(part, js, job);
  J = job_ptr(J, js, job);
  g = job_ptr(g, js, job);
  H = job_ptr(H, js, job);
  cpart = job_ptr(cpart, js, job);
  gmax = job_ptr(gmax, js, job);
  pen = job_ptr(pen, js, job);
  const int s = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (s >= N) return;  // whole warps leave together
  const int St = s / kST, sl = s % kST;
  const int nrow = nS - St, total = nrow + St + 1;
  const int h = lane >> 4, v = lane & 15;
  // the partials of this lane, loaded four at a time (independent loads in
  // flight), added in list order
  double t = 0.0;
  if (v < kRowV) {
    for (int e0 = h; e0 < total; e0 += 8) {
      double x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int e = e0 + 2 * u;
        x[u] = 0.0;
        if (e < nrow) x[u] = part[(size_t)tile_pair(St, St + e, nS) * kPartStride + sl * kRowV + v];
        else if (e < total && v < kColV)
          x[u] = part[(size_t)tile_pair(e - nrow, St, nS) * kPartStride + kST * kRowV + sl * kColV + v];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) t += x[u];
    }
  }
  t += __shfl_down_sync(0xffffffffu, t, 16);
  if (lane < kRowV) {
    const int i = lane;
    if (pen != nullptr) {
      const double* a = pen + 8 * s;
      const double* th = J + 8 * s;
      if (i < 8) {
        t += pen_w * (a[i] - th[i]);
      } else if (i < 10) {
        t += pen_w;
      } else if (i == 12) {
        double e = 0.0;
        for (int k = 0; k < 8; ++k) e += (th[k] - a[k]) * (th[k] - a[k]);
        t += pen_w * e;
      }
    }
    if (i < 8) g[8 * s + i] = t;
    else if (i < 12) H[4 * s + i - 8] = t;
    else cpart[s] = t;
  }
  // max_i |g_s,i| over lanes 0..7, compared as bit patterns
  unsigned long long m = lane < 8 ? ((unsigned long long)__double_as_longlong(t) & 0x7FFFFFFFFFFFFFFFull) : 0ull;
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0 && gmax != nullptr) gmax[s] = __longlong_as_double((long long)m);
}

cudaError_t launch_station_sum(const Shape& s, const double* part, const double* J, double* g, double* H,
                               double* cpart, double* gmax, const LMState* lm, const double* pen, double pen_w,
                               cudaStream_t st, const Batch& bt) {
  const int nS = (s.N + kST - 1) / kST;
  const unsigned blocks = (unsigned)((s.N + kSumThreads / 32 - 1) / (kSumThreads / 32));
  const dim3 grd(blocks, 1, bt.G);
  k_station_sum<<<grd, kSumThreads, 0, st>>>(s.N, nS, part, J, g, H, cpart, gmax, lm, pen, pen_w, bt.js);
  return cudaGetLastError();
}

}  // namespace sc
