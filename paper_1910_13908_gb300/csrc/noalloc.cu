// sc_residual_noalloc: the residual-and-cost call for callers that cannot
// allocate device memory and so cannot hand the library a workspace.
//
// Typical such callers are plug-ins running inside a host application whose
// own allocator already owns the whole device and exposes no way to borrow
// from it, and latency-bound loops that forbid cudaMalloc after start-up
// because an allocation can synchronise the device.  This entry point keeps
// its scratch (the per-baseline partial costs and gradient sums that the
// streaming pass writes before they are summed into the cost) in one
// fixed-size array compiled into the library, so the call itself allocates
// nothing.
//
// Costs of the design, for the user:
//  * every GPU on which the library's device code is loaded holds
//    kScratchBytes of device memory until the process exits.  With CUDA's
//    default lazy module loading that happens at the first call of this
//    entry point on the device (its address lookup loads the module), with
//    CUDA_MODULE_LOADING=EAGER when the context is created; either way it is
//    the one allocation this design makes, so a caller whose allocator later
//    reserves the device should make its first call before that;
//  * all calls on one device share that array, so two calls that overlap on
//    the GPU (other streams, other host threads) race and corrupt each
//    other's cost; serialise them;
//  * problems whose scratch would exceed the array are rejected with
//    SC_EINVAL before anything is launched.
// Every scratch entry the call reads is written earlier in the same call, so
// nothing has to be cleared between calls.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "sc_common.cuh"

namespace sc {

namespace {

constexpr size_t kScratchBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

// The scratch itself.  In host code its name is only a stand-in for the
// device copy: the kernels must be given the address from
// cudaGetSymbolAddress, never &g_scratch.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

thread_local char g_nmsg[256] = "";

// Device address of g_scratch in the current context.  A module global has
// its own address in every CUDA context (a new primary context after
// cudaDeviceReset, or a driver-API context made current by a host
// application), so the address is looked up again on every call made
// outside stream capture.  During capture the address found by the last
// call outside capture on this device is used (a lookup could load the
// module, which is not stream work); with no such call yet the lookup is
// tried once all the same.
int scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    snprintf(g_nmsg, sizeof(g_nmsg), "sc_residual_noalloc: no usable current device (%s)",
             e != cudaSuccess ? cudaGetErrorString(e) : "device ordinal out of range");
    return SC_ECUDA;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) cs = cudaStreamCaptureStatusNone;
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone || g_addr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || p == nullptr) {
      snprintf(g_nmsg, sizeof(g_nmsg),
               "sc_residual_noalloc: cannot find its built-in scratch on device %d (cudaGetSymbolAddress: %s)",
               dev, e != cudaSuccess ? cudaGetErrorString(e) : "null address");
      return SC_ECUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return SC_OK;
}

template <typename R>
int residual_noalloc(const Shape& s, const void* X, const void* C, const double* jones, void* Rout,
                     double* cost, cudaStream_t st) {
  // one chunk holding every timeslot: one (cost, 8 gradient sums) entry per baseline
  const int nchunk = 1, tchunk = s.T;
  size_t need = (size_t)s.B * 9 * sizeof(R);
  if (cost != nullptr && need + 256 > kScratchBytes) {
    snprintf(g_nmsg, sizeof(g_nmsg),
             "sc_residual_noalloc: %lld baselines need %zu bytes of scratch, the built-in limit is %zu "
             "(at most %zu baselines)", (long long)s.B, need, kScratchBytes,
             (kScratchBytes - 256) / (9 * sizeof(R)));
    return SC_EINVAL;
  }
  int flags = P_SUB | (Rout ? P_WRITE_R : 0) | (cost ? P_STATS : 0);
  if (!(flags & (P_WRITE_R | P_STATS))) return SC_OK;
  R* stat_cost = nullptr;
  R* stat_rho = nullptr;
  if (cost != nullptr) {
    void* base = nullptr;
    if (scratch_address(st, &base) != SC_OK) return SC_ECUDA;
    stat_cost = static_cast<R*>(base);
    stat_rho = reinterpret_cast<R*>(static_cast<char*>(base) + ((s.B * sizeof(R) + 255) & ~(size_t)255));
  }
  cudaError_t e = launch_pass<R>(s, flags, static_cast<const R*>(X), static_cast<const R*>(C), nullptr, jones,
                                 static_cast<R*>(Rout), stat_cost, stat_rho, nchunk, tchunk, nullptr, st);
  if (e == cudaSuccess && cost != nullptr) e = launch_sum_reals<R>(stat_cost, s.B, cost, st);
  if (e != cudaSuccess) {
    snprintf(g_nmsg, sizeof(g_nmsg), "sc_residual_noalloc: %s", cudaGetErrorString(e));
    return SC_ECUDA;
  }
  return SC_OK;
}

}  // namespace
}  // namespace sc

using namespace sc;

extern "C" SC_API int32_t sc_residual_noalloc(const sc_dims* d, const void* X, const void* C,
                                              const double* jones, void* R, double* cost, int32_t prec,
                                              void* stream, char* errbuf, size_t errlen) {
  g_nmsg[0] = 0;
  int rc = SC_OK;
  if (d == nullptr || (prec != SC_FP64 && prec != SC_MIXED)) {
    snprintf(g_nmsg, sizeof(g_nmsg), "sc_residual_noalloc: bad dims or precision");
    rc = SC_EINVAL;
  } else if (d->N < 2 || d->N > 8000 || d->T < 1 || d->F < 1 || (int64_t)d->T * d->F > 65535) {
    // the same shape limits as sc_residual
    snprintf(g_nmsg, sizeof(g_nmsg),
             "sc_residual_noalloc: N must be in [2, 8000], T and F >= 1 and T*F <= 65535 "
             "(N=%d T=%d F=%d)", d->N, d->T, d->F);
    rc = SC_EINVAL;
  } else if (!X || !C || !jones) {
    snprintf(g_nmsg, sizeof(g_nmsg), "sc_residual_noalloc: X, C and jones must not be NULL");
    rc = SC_EINVAL;
  } else {
    Shape s;
    s.N = d->N;
    s.T = d->T;
    s.F = d->F;
    s.K = 1;
    s.S_max = 0;
    s.B = (int64_t)d->N * (d->N - 1) / 2;
    s.prec = prec;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = prec == SC_MIXED ? residual_noalloc<float>(s, X, C, jones, R, cost, st)
                          : residual_noalloc<double>(s, X, C, jones, R, cost, st);
  }
  if (errbuf != nullptr && errlen > 0) {
    strncpy(errbuf, g_nmsg, errlen - 1);
    errbuf[errlen - 1] = 0;
  }
  return rc;
}
