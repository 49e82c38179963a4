// After calibration: the residual of the whole sky model, optionally
// corrected for the gains of one direction c,
//     R = V - sum_k c_k(t,f) G_k,      G_k = J_kp J_kq^H
//     R <- J_cp^{-1} R J_cq^{-H}
// in one streaming pass.  Every visibility of V is read once, the coherency
// of every cluster once, and R written once: (8K + 64) bytes per visibility
// in SC_MIXED (complex64), twice that in SC_FP64.  Subtracting one cluster
// at a time would stream V and R through HBM K times.
//
// Work item: one baseline and a slab of NV consecutive (timeslot, channel)
// pairs.  Consecutive threads take consecutive baselines of the same slab, so
// a warp's loads of V, C and R cover contiguous [F][2][2] and [F] blocks.
// The NV accumulators stay in registers through the cluster loop; per
// cluster and item the thread loads J_kp and J_kq (a few hundred KB for all
// clusters, L2-resident, rounded to R once by k_gain_prep) and forms G_k once
// for its NV visibilities.  (Channel-major items, one (baseline, channel)
// pair per thread with fully contiguous warp accesses, measured slower: each
// of the F threads of a baseline forms G_k again.)
#include <algorithm>

#include "sc_common.cuh"

namespace sc {

// Jr [K][N][8]: every cluster's Jones rounded to R.  Jinv [N][8]: the
// inverses of cluster corr's Jones, adjugate over determinant in float64,
// then rounded.  A station with |det J|^2 <= 1e-24 |J|_F^4 (that is
// |det J| <= 1e-12 |J|_F^2) gets Jinv = 0, which zeroes its baselines, and
// raises SC_STATUS_SINGULAR.
template <typename R>
__global__ void k_gain_prep(int K, int N, int corr, const double* __restrict__ J,
                            R* __restrict__ Jr, R* __restrict__ Jinv,
                            uint32_t* __restrict__ status) {
  const int KN = K * N;
  const int n = KN + (corr >= 0 ? N : 0);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (i < KN) {
#pragma unroll
      for (int e = 0; e < 8; ++e) Jr[8 * (size_t)i + e] = (R)J[8 * (size_t)i + e];
      continue;
    }
    const int s = i - KN;
    const double* g = J + 8 * ((size_t)corr * N + s);
    const cx<double> a{g[0], g[1]}, b{g[2], g[3]}, c{g[4], g[5]}, d{g[6], g[7]};
    const cx<double> det = a * d - b * c;
    const double fro2 = norm2(a) + norm2(b) + norm2(c) + norm2(d);
    R* o = Jinv + 8 * (size_t)s;
    if (norm2(det) <= 1e-24 * fro2 * fro2) {
#pragma unroll
      for (int e = 0; e < 8; ++e) o[e] = (R)0;
      atomicOr(status, SC_STATUS_SINGULAR);
      continue;
    }
    // 1/det = conj(det) / |det|^2
    const cx<double> r = scale(conj(det), 1.0 / norm2(det));
    const cx<double> nb{-b.re, -b.im}, nc{-c.re, -c.im};
    const cx<double> v[4] = {d * r, nb * r, nc * r, a * r};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      o[2 * e] = (R)v[e].re;
      o[2 * e + 1] = (R)v[e].im;
    }
  }
}

// one visibility by coherent (not read-only-path) vector loads, since R may
// be V
__device__ __forceinline__ m22<float> ld_vis_rw(const float* p) {
  const float4 u = reinterpret_cast<const float4*>(p)[0], v = reinterpret_cast<const float4*>(p)[1];
  return {{u.x, u.y}, {u.z, u.w}, {v.x, v.y}, {v.z, v.w}};
}
__device__ __forceinline__ m22<double> ld_vis_rw(const double* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = q[0], b = q[1], c = q[2], d = q[3];
  return {{a.x, a.y}, {b.x, b.y}, {c.x, c.y}, {d.x, d.y}};
}

// Per data type: NV visibilities per work item, the unroll of the cluster
// loop and the blocks per SM the register budget is cut for.  For complex64,
// 4 visibilities with the loop unrolled 4 times keep 16 coherency loads of
// each thread in flight at 128 registers, 2 blocks of 256 per SM (64 KB of
// loads per SM; an HBM stream needs about half that).  The float64 path, kept
// for comparison, uses 1 block per SM without spills.
template <typename R> struct SlabOf;
template <> struct SlabOf<float> {
  static constexpr int NV = 4, UNROLL = 4, MINB = 2;
};
template <> struct SlabOf<double> {
  static constexpr int NV = 4, UNROLL = 1, MINB = 1;
};

// IX: index type of a visibility or coherency element; uint32_t when
// 2 K T B F < 2^31 (every index into C fits), else size_t.
template <typename R, int NV, typename IX>
__global__ void __launch_bounds__(256, SlabOf<R>::MINB) k_residual_all(int N, int T, int F, int64_t B, int K,
                                                      int nslab, const R* V,
                                                      const R* __restrict__ C,
                                                      const R* __restrict__ Jr,
                                                      const R* __restrict__ Jinv, R* Rout,
                                                      double* __restrict__ part) {
  const int TF = T * F;
  const int64_t n_items = (int64_t)nslab * B;
  const IX per_cluster = (IX)TF * (IX)B;  // T*B*F coherencies
  double cost = 0.0;
  // grid-stride over (slab, baseline) items; the grid is sized to the
  // resident blocks
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < n_items;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int slab = (int)(idx / B);
    const int64_t b = idx - (int64_t)slab * B;
    int p, q;
    bl_pair(b, N, p, q);
    const int r0 = slab * NV;
    const int nv = min(NV, TF - r0);
    // visibility index (t*B + b)*F + f of the slab's pairs r0 .. r0+NV-1
    IX off[NV];
    {
      int t = r0 / F, f = r0 - t * F;
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        off[i] = ((IX)t * (IX)B + (IX)b) * (IX)F + (IX)f;
        if (++f == F) {
          f = 0;
          ++t;
        }
      }
    }
    m22<R> acc[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      acc[i] = i < nv ? ld_vis_rw(V + 8 * off[i]) : mzero<R>();
    }
#pragma unroll(SlabOf<R>::UNROLL)
    for (int k = 0; k < K; ++k) {
      const m22<R> G = mul_h(ld_vis(Jr + 8 * ((size_t)k * N + p)), ld_vis(Jr + 8 * ((size_t)k * N + q)));
      const R* Ck = C + (IX)2 * (IX)k * per_cluster;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < nv) acc[i] = acc[i] - smul(ld_c(Ck + 2 * off[i]), G);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) cost += (double)frob2(acc[i]);
    if (Jinv != nullptr) {
      const m22<R> Ip = ld_vis(Jinv + 8 * (size_t)p), Iq = ld_vis(Jinv + 8 * (size_t)q);
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = mul_h(mul(Ip, acc[i]), Iq);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) st_vis(Rout + 8 * off[i], acc[i]);
  }
  if (part == nullptr) return;
  // block sum of the cost, in a fixed order for a fixed grid
  __shared__ double sh[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = cost;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

// ---- complex64: coherencies staged through a shared-memory ring ------------------------
//
// The register kernel above keeps one cluster's NV coherency loads of each
// thread in flight: about 16 KB per SM, well short of what HBM latency
// needs.  Here every thread streams its own (item, cluster) sequence
// through a ring of S stages in shared memory filled by cp.async, with a
// prefetch cursor S steps ahead of the arithmetic (crossing item
// boundaries), so S x NV x 8 B of each thread are in flight without holding
// registers.  The visibilities of an item arrive with its first stage.  A
// thread reads only slots it filled itself, so cp.async.wait_group alone
// orders the data (no block barrier).  Slots are laid out [stage][i][thread]
// so a warp's 8-byte reads are conflict-free.  Requires K >= S: the
// visibility slot of an item is refilled only after its first stage has
// been consumed.

namespace {
__device__ __forceinline__ void ra_cp8(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ra_cp16(void* dst, const void* src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void ra_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int W>
__device__ __forceinline__ void ra_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(W) : "memory"); }
}  // namespace

constexpr int kPipeNV = 4;     // visibilities per item
constexpr int kPipeThreads = 256;

template <int S>
constexpr size_t pipe_smem_bytes() {
  return (size_t)S * kPipeNV * kPipeThreads * 8 + (size_t)kPipeNV * 2 * kPipeThreads * 16;
}

template <typename IX, int S>
__global__ void __launch_bounds__(kPipeThreads, 2) k_residual_all_pipe(
    int N, int T, int F, int64_t B, int K, int nslab, const float* V, const float* __restrict__ C,
    const float* __restrict__ Jr, const float* __restrict__ Jinv, float* Rout,
    double* __restrict__ part) {
  constexpr int NV = kPipeNV;
  extern __shared__ __align__(16) unsigned char ra_smem[];
  float2* ring = reinterpret_cast<float2*>(ra_smem);                                  // [S][NV][T]
  float4* vslot = reinterpret_cast<float4*>(ra_smem + (size_t)S * NV * kPipeThreads * 8);  // [2NV][T]
  const int tid = threadIdx.x;
  const int TF = T * F;
  const int64_t n_items = (int64_t)nslab * B;
  const int64_t stride = (int64_t)gridDim.x * kPipeThreads;
  const IX per_cluster = (IX)TF * (IX)B;

  // visibility offsets (t*B + b)*F + f of item idx's NV (t, f) pairs
  auto offsets = [&](int64_t idx, IX* off, int& nv) {
    const int slab = (int)(idx / B);
    const int64_t b = idx - (int64_t)slab * B;
    const int r0 = slab * NV;
    nv = min(NV, TF - r0);
    int t = r0 / F, f = r0 - t * F;
#pragma unroll
    for (int i = 0; i < NV; ++i) {
      off[i] = ((IX)t * (IX)B + (IX)b) * (IX)F + (IX)f;
      if (++f == F) {
        f = 0;
        ++t;
      }
    }
  };

  // prefetch cursor: (pf_idx, pf_k), S steps ahead of the arithmetic
  int64_t pf_idx = (int64_t)blockIdx.x * kPipeThreads + tid;
  int pf_k = 0, pf_nv = 0, pf_stage = 0;
  IX pf_off[NV];
  if (pf_idx < n_items) offsets(pf_idx, pf_off, pf_nv);
  auto issue = [&]() {
    if (pf_idx < n_items) {
      const float* Ck = C + (IX)2 * (IX)pf_k * per_cluster;
#pragma unroll
      for (int i = 0; i < NV; ++i)
        if (i < pf_nv) ra_cp8(&ring[((size_t)pf_stage * NV + i) * kPipeThreads + tid], Ck + 2 * pf_off[i]);
      if (pf_k == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i)
          if (i < pf_nv) {
            ra_cp16(&vslot[(2 * i) * kPipeThreads + tid], V + 8 * pf_off[i]);
            ra_cp16(&vslot[(2 * i + 1) * kPipeThreads + tid], V + 8 * pf_off[i] + 4);
          }
      }
    }
    ra_commit();
    pf_stage = pf_stage + 1 == S ? 0 : pf_stage + 1;
    if (++pf_k == K) {
      pf_k = 0;
      pf_idx += stride;
      if (pf_idx < n_items) offsets(pf_idx, pf_off, pf_nv);
    }
  };
#pragma unroll 1
  for (int s = 0; s < S; ++s) issue();

  double cost = 0.0;
  int stage = 0;
#pragma unroll 1
  for (int64_t idx = (int64_t)blockIdx.x * kPipeThreads + tid; idx < n_items; idx += stride) {
    IX off[NV];
    int nv;
    offsets(idx, off, nv);
    const int64_t b = idx % B;
    int p, q;
    bl_pair(b, N, p, q);
    m22<float> acc[NV];
    m22<float> Jp = ld_vis(Jr + 8 * (size_t)p), Jq = ld_vis(Jr + 8 * (size_t)q);
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
      const m22<float> G = mul_h(Jp, Jq);
      if (k + 1 < K) {
        Jp = ld_vis(Jr + 8 * ((size_t)(k + 1) * N + p));
        Jq = ld_vis(Jr + 8 * ((size_t)(k + 1) * N + q));
      }
      ra_wait<S - 1>();
      if (k == 0) {
#pragma unroll
        for (int i = 0; i < NV; ++i) {
          const float4 u = vslot[(2 * i) * kPipeThreads + tid], w = vslot[(2 * i + 1) * kPipeThreads + tid];
          acc[i] = {{u.x, u.y}, {u.z, u.w}, {w.x, w.y}, {w.z, w.w}};
        }
      }
#pragma unroll
      for (int i = 0; i < NV; ++i) {
        const float2 c = ring[((size_t)stage * NV + i) * kPipeThreads + tid];
        acc[i] = acc[i] - smul(cx<float>{c.x, c.y}, G);
      }
      stage = stage + 1 == S ? 0 : stage + 1;
      issue();
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) cost += (double)frob2(acc[i]);
    if (Jinv != nullptr) {
      const m22<float> Ip = ld_vis(Jinv + 8 * (size_t)p), Iq = ld_vis(Jinv + 8 * (size_t)q);
#pragma unroll
      for (int i = 0; i < NV; ++i) acc[i] = mul_h(mul(Ip, acc[i]), Iq);
    }
#pragma unroll
    for (int i = 0; i < NV; ++i)
      if (i < nv) st_vis(Rout + 8 * off[i], acc[i]);
  }
  ra_wait<0>();
  if (part == nullptr) return;
  __shared__ double sh[kPipeThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cost += __shfl_xor_sync(0xffffffffu, cost, o);
  if ((tid & 31) == 0) sh[tid >> 5] = cost;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kPipeThreads / 32; ++w) t += sh[w];
    part[blockIdx.x] = t;
  }
}

template <typename R>
cudaError_t launch_gain_prep(const Shape& s, const double* J, int corr, R* Jr, R* Jinv,
                             uint32_t* status, cudaStream_t st) {
  const int n = s.K * s.N + (corr >= 0 ? s.N : 0);
  k_gain_prep<R><<<(n + 255) / 256, 256, 0, st>>>(s.K, s.N, corr, J, Jr, Jinv, status);
  return cudaGetLastError();
}

constexpr int kPipeStages = 4;

// resident blocks of a kernel at the given block size and dynamic shared memory
template <typename Kern>
static int resident_blocks(Kern kern, int threads, size_t smem) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, threads, smem);
  return std::max(1, sms * std::max(per, 1));
}

template <typename IX>
static cudaError_t go_pipe(const Shape& s, const float* V, const float* C, const float* Jr,
                          const float* Jinv, float* Rout, double* part, int max_parts, int* n_parts,
                          cudaStream_t st) {
  constexpr int S = kPipeStages;
  constexpr size_t smem = pipe_smem_bytes<S>();
  // per device and cheap: set on every launch
  cudaError_t e = cudaFuncSetAttribute(k_residual_all_pipe<IX, S>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  static const int resident = resident_blocks(k_residual_all_pipe<IX, S>, kPipeThreads, smem);
  const int nslab = (s.T * s.F + kPipeNV - 1) / kPipeNV;
  const int64_t n_items = (int64_t)nslab * s.B;
  const int grid = (int)std::min<int64_t>(
      std::min<int64_t>((n_items + kPipeThreads - 1) / kPipeThreads, resident), max_parts);
  k_residual_all_pipe<IX, S><<<grid, kPipeThreads, smem, st>>>(s.N, s.T, s.F, s.B, s.K, nslab, V, C, Jr,
                                                               Jinv, Rout, part);
  *n_parts = grid;
  return cudaGetLastError();
}

template <typename R>
cudaError_t launch_residual_all(const Shape& s, const R* V, const R* C, const R* Jr,
                                const R* Jinv, R* Rout, double* part, int max_parts, int* n_parts,
                                cudaStream_t st) {
  constexpr int NV = SlabOf<R>::NV;
  const uint64_t top_ = (uint64_t)s.T * s.F * (uint64_t)s.B * (uint64_t)std::max(8, 2 * s.K);
  if constexpr (sizeof(R) == 4) {
    if (s.K >= kPipeStages) {
      return top_ < (1ull << 31)
                 ? go_pipe<uint32_t>(s, V, C, Jr, Jinv, Rout, part, max_parts, n_parts, st)
                 : go_pipe<size_t>(s, V, C, Jr, Jinv, Rout, part, max_parts, n_parts, st);
    }
  }
  static const int resident = [] {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_residual_all<R, NV, uint32_t>, 256, 0);
    return std::max(1, sms * std::max(per, 1));
  }();
  const int nslab = (s.T * s.F + NV - 1) / NV;
  const int64_t n_items = (int64_t)nslab * s.B;
  const int grid =
      (int)std::min<int64_t>(std::min<int64_t>((n_items + 255) / 256, resident), max_parts);
  // largest index: 8 T B F (V, R) or 2 K T B F (C)
  const uint64_t top = (uint64_t)s.T * s.F * (uint64_t)s.B * (uint64_t)std::max(8, 2 * s.K);
  if (top < (1ull << 31))
    k_residual_all<R, NV, uint32_t><<<grid, 256, 0, st>>>(s.N, s.T, s.F, s.B, s.K, nslab, V, C, Jr,
                                                          Jinv, Rout, part);
  else
    k_residual_all<R, NV, size_t><<<grid, 256, 0, st>>>(s.N, s.T, s.F, s.B, s.K, nslab, V, C, Jr,
                                                        Jinv, Rout, part);
  *n_parts = grid;
  return cudaGetLastError();
}

#define SC_INST(R)                                                                              \
  template cudaError_t launch_gain_prep<R>(const Shape&, const double*, int, R*, R*, uint32_t*, \
                                           cudaStream_t);                                       \
  template cudaError_t launch_residual_all<R>(const Shape&, const R*, const R*, const R*,       \
                                              const R*, R*, double*, int, int*, cudaStream_t);
SC_INST(float)
SC_INST(double)
#undef SC_INST

}  // namespace sc
