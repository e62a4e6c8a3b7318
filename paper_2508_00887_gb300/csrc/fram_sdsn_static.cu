// fram_sdsn_static: the SDSN entry point for callers that cannot allocate
// device memory.
//
// Some callers must not have a library call cudaMalloc/cudaFree behind their
// back: applications whose device memory is owned by another allocator (a
// framework's caching allocator or a pool reserved up front, where a foreign
// cudaMalloc breaks the memory accounting or fails because the pool holds
// everything), and latency-bound loops for which the implicit device-wide
// synchronisation of cudaFree is not acceptable.  This entry point runs the
// same SDSN kernel as fram_sdsn, with the same launch configuration, but takes
// all of its scratch (row/column/tile partials, grid barrier, max(X), status)
// from one file-scope static device array.  It creates no context and calls
// no allocating routine.
//
// Properties of the static array:
//  * its size is fixed at build time (kStaticBytes below, about 2 MiB); it
//    bounds n at FRAM_SDSN_STATIC_MAX_N and is held on every GPU that loads
//    this library until the process exits;
//  * every call on a device shares it and it keeps the last call's contents:
//    the barrier, the max(X) key and the status are cleared at the start of
//    each call, and the partials are fully rewritten before they are read;
//  * calls whose work overlaps on the GPU (different streams, or different
//    host threads on the same device) race on it and give undefined results.
//    Serialise them on one stream.
//
// In host code the array's name is only a host-side stand-in, not a device
// address.  The device address is looked up once per device with
// cudaGetSymbolAddress, with that device current, on the first call made on
// that device; that first call should therefore come before any stream
// capture begins.
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/fram.h"
#include "fram_internal.cuh"

namespace {

using namespace fram;

// Header (stats, barrier, max key) then the SDSN partials for n up to
// FRAM_SDSN_STATIC_MAX_N on grids of up to 16 x 16 CTAs.
constexpr int kMaxGridSide = 16;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kPartialDoubles =
    (size_t)4 * kMaxGridSide * FRAM_SDSN_STATIC_MAX_N + 2 * kMaxGridSide * kMaxGridSide + 64;
constexpr size_t kStaticBytes = kHeaderBytes + kPartialDoubles * sizeof(double);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticHeader {
  SdsnStats stats;
  GridBarrier barrier;
  unsigned long long xmax_key;
};
static_assert(sizeof(StaticHeader) <= kHeaderBytes, "header does not fit");

std::mutex g_setup_mu;
unsigned char* g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

void put_err(char* err, size_t len, const char* msg, const char* detail = "") {
  if (err && len) snprintf(err, len, "%s%s", msg, detail);
}

fram_status cuda_err(char* err, size_t len, const char* what, cudaError_t e) {
  if (e == cudaSuccess) {  // refused by a launch limit, not by a CUDA call
    if (err && len)
      snprintf(err, len, "%s: the launch exceeds this GPU's limits (co-resident CTAs or shared "
                         "memory) for this problem size", what);
    return FRAM_ERR_INVALID;
  }
  if (err && len) snprintf(err, len, "%s: %s", what, cudaGetErrorString(e));
  cudaGetLastError();
  return FRAM_ERR_CUDA;
}

}  // namespace

extern "C" fram_status fram_sdsn_static(int n, const double* X, double* D, double theta,
                                        double gamma_tol, int max_sweeps, void* cuda_stream,
                                        int* sweeps_out, double* gamma_out, char* err,
                                        size_t err_len) {
  if (err && err_len) err[0] = '\0';
  if (n < 1 || X == nullptr || D == nullptr || !(theta > 0.0) || max_sweeps < 1) {
    put_err(err, err_len, "fram_sdsn_static: n >= 1, non-NULL X and D, theta > 0 and "
                          "max_sweeps >= 1 are required");
    return FRAM_ERR_INVALID;
  }
  if (n > FRAM_SDSN_STATIC_MAX_N) {
    char d[96];
    snprintf(d, sizeof d, " (n = %d, limit %d)", n, FRAM_SDSN_STATIC_MAX_N);
    put_err(err, err_len, "fram_sdsn_static: n exceeds the static scratch limit", d);
    return FRAM_ERR_INVALID;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(err, err_len, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    put_err(err, err_len, "fram_sdsn_static: device index out of range");
    return FRAM_ERR_INVALID;
  }
  unsigned char* base;
  int num_sms;
  {
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (g_scratch_addr[dev] == nullptr) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess) return cuda_err(err, err_len, "cudaGetSymbolAddress", e);
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_err(err, err_len, "cudaDeviceGetAttribute", e);
      g_num_sms[dev] = sms;
      g_scratch_addr[dev] = static_cast<unsigned char*>(p);
    }
    base = g_scratch_addr[dev];
    num_sms = g_num_sms[dev];
  }
  if (sdsn_partials_elems(n, num_sms) > kPartialDoubles) {
    put_err(err, err_len, "fram_sdsn_static: this GPU's SDSN grid needs more scratch than the "
                          "static array holds");
    return FRAM_ERR_INVALID;
  }
  StaticHeader* h = reinterpret_cast<StaticHeader*>(base);
  double* partials = reinterpret_cast<double*>(base + kHeaderBytes);

  // The array keeps the previous call's contents: clear what must start at 0.
  e = cudaMemsetAsync(h, 0, sizeof(StaticHeader), s);
  if (e != cudaSuccess) return cuda_err(err, err_len, "cudaMemsetAsync", e);
  if (launch_max(X, n, n, &h->xmax_key, s) < 0)
    return cuda_err(err, err_len, "max kernel", cudaGetLastError());
  SdsnLaunch L{};
  L.n = n;
  L.X = X;
  L.ldx = n;
  L.Y = D;
  L.ldy = n;
  L.theta = theta;
  L.gamma_tol = gamma_tol;
  L.max_sweeps = max_sweeps;
  L.xmax_key = &h->xmax_key;
  L.stats = &h->stats;
  L.partials = partials;
  L.barrier = &h->barrier;
  L.limit_ns = kWaitLimitNs;
  if (launch_sdsn_fp64(L, num_sms, s) < 0)
    return cuda_err(err, err_len, "sdsn kernel", cudaGetLastError());
  SdsnStats st;
  e = cudaMemcpyAsync(&st, &h->stats, sizeof st, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_err(err, err_len, "readback", e);
  if (st.status == DEV_DEGENERATE) {
    put_err(err, err_len, "fram_sdsn_static: max(X) <= 0, SDSN step 1 is undefined");
    return FRAM_ERR_DEGENERATE;
  }
  if (st.status != DEV_OK) {
    put_err(err, err_len, "fram_sdsn_static: a device-side wait exceeded its limit");
    return FRAM_ERR_TIMEOUT;
  }
  if (sweeps_out) *sweeps_out = st.sweeps;
  if (gamma_out) *gamma_out = st.gamma;
  return FRAM_OK;
}
