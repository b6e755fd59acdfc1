// sip_project_l1_noalloc: the l1-ball projection of sip_project_set, run
// without any allocation.  Everything the projection needs beyond the
// caller's input and output (the work list, the selection job's state and
// its radix histograms) lives in one file-scope device array compiled into
// the library.
//
// Who needs this: callers that must not allocate device memory while they
// run.  Examples: code running under a memory pool or budget that a raw
// cudaMalloc would bypass or overcommit, and latency-sensitive loops where
// cudaMalloc / cudaFree may synchronise the device and stall other work.
//
// Costs of the fixed array: it holds kNoAllocBytes on every GPU that loads
// the library, for as long as the library stays loaded.  Every call on a
// device reuses the same array, so calls whose device work overlaps (two
// streams, or two host threads on one device) race and must be serialised
// by the caller.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda_runtime.h>

#include "sip.h"
#include "sip_dev.cuh"
#include "sip_host.h"
#include "sip_kernels.h"

namespace sip {
namespace {

constexpr int kNoAllocTiles = 1024;

// Layout of the scratch array.
struct NoAllocScratch {
  InstDev inst;
  InstScal scal;
  JobDev job;
  JobScal jscal;
  Tile tiles[kNoAllocTiles];
  uint32_t hcnt[kBins];
  double hs1[kBins], hs2[kBins], hs3[kBins];
  double l1;          // ||w||_1 (binary64)
  uint32_t arrive;    // CTAs done in the norm kernel
  uint32_t nonfinite; // ||w||_1 is not finite: w holds a NaN or an infinity
};

constexpr size_t kNoAllocBytes = (sizeof(NoAllocScratch) + 255) / 256 * 256;

// The scratch: file scope, 256-byte aligned, allocated with the module.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

__device__ __forceinline__ double na_warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ||w||_1 in binary64 over the whole vector; the last CTA arms the
// selection job exactly as the set pass does for an l1 set: the radius tau,
// and JM_NONE (tau = 0), JM_ALL (w already inside the ball) or JM_SELECT.
template <typename T>
__global__ void __launch_bounds__(256) k_na_l1norm(const T *__restrict__ w, int64_t n, NoAllocScratch *S,
                                                   double tau) {
  double part = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    part += fabs((double)w[i]);
  __shared__ double sm[8];
  part = na_warp_sum(part);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = part;
  __syncthreads();
  __shared__ bool last;
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sm[i];
    atomicAdd(&S->l1, t);
    __threadfence();
    last = atomicAdd(&S->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last || threadIdx.x != 0) return;
  __threadfence();
  const double l1 = *(volatile double *)&S->l1;
  JobScal &js = S->jscal;
  S->nonfinite = isfinite(l1) ? 0u : 1u;
  js.active = 1;
  js.pass = 0;
  js.prefix = 0;
  js.n_above = 0;
  js.c_above = js.s1_above = js.s2_above = 0.0;
  js.tie_needed = 0;
  js.counter = 0;
  js.tau = tau;
  js.theta = 0.0;
  js.thetaf = 0.f;
  // a non-finite norm has no threshold: no selection pass runs and the
  // output is NaN
  js.mode = !isfinite(l1) || tau == 0.0 ? JM_NONE : (l1 <= tau ? JM_ALL : JM_SELECT);
}

// y = sign(w) max(|w| - theta, 0), the arithmetic of the final pass.
template <typename T>
__global__ void k_na_soft(const T *__restrict__ w, T *__restrict__ y, int64_t n, const NoAllocScratch *S) {
  const JobScal &js = S->jscal;
  const int mode = js.mode;
  const bool bad = S->nonfinite != 0u;
  const T th = sizeof(T) == 4 ? (T)js.thetaf : (T)js.theta;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const T wv = w[i];
    T yn;
    if (bad) {
      yn = T(NAN);
    } else if (mode == JM_ALL) {
      yn = wv;
    } else if (mode == JM_NONE) {
      yn = T(0);
    } else {
      const T a = fabs(wv) - th;
      yn = a > T(0) ? copysign(a, wv) : T(0);
    }
    y[i] = yn;
  }
}

// Device address of the scratch and the SM count, fetched once per device
// with that device current (a host-side reference to the array's name is
// not a device address).
std::mutex g_na_mutex;
void *g_na_addr[kMaxDevices] = {};
int g_na_sms[kMaxDevices] = {};

sip_status scratch_address(NoAllocScratch **out, int *sms) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return fail(SIP_ERR_CUDA, "cudaGetDevice failed");
  }
  if (dev < 0 || dev >= kMaxDevices) return fail(SIP_ERR_INTERNAL, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return fail(SIP_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    }
    int n_sm = 0;
    e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess || n_sm < 1) {
      cudaGetLastError();
      return fail(SIP_ERR_CUDA, "SM count: %s", cudaGetErrorString(e));
    }
    if (cudaError_t e2 = kernels_setup()) return fail(SIP_ERR_CUDA, "kernel set-up: %s", cudaGetErrorString(e2));
    g_na_sms[dev] = n_sm;
    g_na_addr[dev] = p;
  }
  *out = (NoAllocScratch *)g_na_addr[dev];
  *sms = g_na_sms[dev];
  return SIP_OK;
}

}  // namespace
}  // namespace sip

using namespace sip;

extern "C" sip_status sip_project_l1_noalloc(int dtype, const void *w_dev, int64_t n, double tau, void *y_dev,
                                             void *stream, double *theta_out) {
  if (!w_dev || !y_dev) return fail(SIP_ERR_INVALID_ARG, "NULL buffer");
  if (dtype != SIP_F64 && dtype != SIP_F32) return fail(SIP_ERR_INVALID_ARG, "unknown dtype");
  if (n < 1) return fail(SIP_ERR_INVALID_ARG, "n must be >= 1");
  if (n > SIP_NOALLOC_MAX_N)
    return fail(SIP_ERR_INVALID_ARG, "n = %lld exceeds SIP_NOALLOC_MAX_N = %lld (the fixed scratch size)",
                (long long)n, (long long)SIP_NOALLOC_MAX_N);
  if (!(tau >= 0.0) || !std::isfinite(tau)) return fail(SIP_ERR_INVALID_ARG, "tau must be finite and >= 0");
  NoAllocScratch *S = nullptr;
  int sms = 0;
  sip_status st = scratch_address(&S, &sms);
  if (st) return st;
  cudaStream_t cs = (cudaStream_t)stream;

  // Descriptors of one 1 x n instance and one l1 selection job over w.
  InstDev d;
  memset(&d, 0, sizeof d);
  d.nz = (int32_t)n;
  d.nx = d.ny = 1;
  d.ndim = 2;
  set_fastdiv(d);
  d.N = n;
  d.nb = d.p = 1;
  d.w = const_cast<void *>(w_dev);  // read only by the selection kernel
  InstScal sc;
  memset(&sc, 0, sizeof sc);        // done = 0: the selection passes run
  JobDev jd;
  memset(&jd, 0, sizeof jd);
  jd.kind = JOB_L1;
  jd.M = n;
  // about one wave: three CTAs per SM (the selection kernel's occupancy)
  const int64_t wave = 3 * (int64_t)sms;
  int64_t chunk = (n + kNoAllocTiles - 1) / kNoAllocTiles;
  const int64_t even = (n + wave - 1) / wave;
  if (chunk < even) chunk = even;
  chunk = (chunk + 255) / 256 * 256;
  Tile tiles[kNoAllocTiles];
  int nt = 0;
  for (int64_t s = 0; s < n; s += chunk, ++nt) {
    tiles[nt].inst = 0;
    tiles[nt].item = 0;
    tiles[nt].start = s;
    tiles[nt].len = (int32_t)(n - s < chunk ? n - s : chunk);
    tiles[nt].seq = nt;
  }
  jd.ntiles = nt;

#define NA_CK(call)                                                                            \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) return fail(SIP_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)
  // the array keeps the previous call's contents: reset what must start at 0
  NA_CK(cudaMemsetAsync(S, 0, sizeof(NoAllocScratch), cs));
  NA_CK(cudaMemcpyAsync(&S->inst, &d, sizeof d, cudaMemcpyHostToDevice, cs));
  NA_CK(cudaMemcpyAsync(&S->scal, &sc, sizeof sc, cudaMemcpyHostToDevice, cs));
  NA_CK(cudaMemcpyAsync(&S->job, &jd, sizeof jd, cudaMemcpyHostToDevice, cs));
  NA_CK(cudaMemcpyAsync(S->tiles, tiles, nt * sizeof(Tile), cudaMemcpyHostToDevice, cs));
  const unsigned grid = (unsigned)((n + 255) / 256 < wave ? (n + 255) / 256 : wave);
  if (dtype == SIP_F64)
    k_na_l1norm<double><<<grid, 256, 0, cs>>>((const double *)w_dev, n, S, tau);
  else
    k_na_l1norm<float><<<grid, 256, 0, cs>>>((const float *)w_dev, n, S, tau);
  NA_CK(cudaGetLastError());
  const Launch L{dtype, cs};
  for (int pass = 0; pass < select_passes(dtype); ++pass)
    NA_CK(launch_select(L, S->tiles, nt, &S->inst, &S->scal, &S->job, &S->jscal, S->hcnt, S->hs1, S->hs2, S->hs3,
                        0, pass, InstOne{}));  // one histogram buffer, cleared by each pass's last CTA
  if (dtype == SIP_F64)
    k_na_soft<double><<<grid, 256, 0, cs>>>((const double *)w_dev, (double *)y_dev, n, S);
  else
    k_na_soft<float><<<grid, 256, 0, cs>>>((const float *)w_dev, (float *)y_dev, n, S);
  NA_CK(cudaGetLastError());
  if (theta_out) {
    JobScal js;
    uint32_t bad = 0;
    NA_CK(cudaMemcpyAsync(&js, &S->jscal, sizeof js, cudaMemcpyDeviceToHost, cs));
    NA_CK(cudaMemcpyAsync(&bad, &S->nonfinite, sizeof bad, cudaMemcpyDeviceToHost, cs));
    NA_CK(cudaStreamSynchronize(cs));
    if (bad) {
      *theta_out = NAN;
      return fail(SIP_ERR_NONFINITE, "w holds a NaN or an infinity (||w||_1 is not finite)");
    }
    *theta_out = js.mode == JM_SELECT ? js.theta : 0.0;
  }
#undef NA_CK
  return SIP_OK;
}
