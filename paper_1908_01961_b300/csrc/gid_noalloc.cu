// Base-colour refinement step for callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc: code running inside another framework's
// memory pool (which forbids raw device allocations or would fragment), real-time
// loops that may not block on the allocator, or host processes that only receive
// device pointers from someone else.  gid_dense_refine_noalloc() runs the same
// k_dense kernel as gid_run's base-colour step, but takes its scratch (block
// partials, completion counter, the K x K systems and the colour table) from the
// file-scope array below instead of a context.  The caller passes the inputs and
// the outputs; the library allocates nothing.
//
// The array is a static __device__ symbol: every GPU that loads this library
// holds GID_NOALLOC_SCRATCH_BYTES of it until the process exits.  In host code
// its name is only a stand-in, so the host asks the runtime for its device
// address once per device (cudaGetSymbolAddress, with that device current).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/gid.h"

// The shared header also defines the frame kernels that gid.cu launches; give
// this translation unit's copies other names so the two objects link together.
#define k_ingest k_ingest_noalloc_tu
#define k_prior_weights k_prior_weights_noalloc_tu
#define k_reset_colors k_reset_colors_noalloc_tu
#define k_relabel k_relabel_noalloc_tu
#include "gid_kernels.cuh"
#undef k_ingest
#undef k_prior_weights
#undef k_reset_colors
#undef k_relabel

using namespace gid;

namespace {

constexpr int kMaxDenseBlocks = 296;                                   // at most 296 row-striding blocks
constexpr int kMaxAcc = GID_MAX_K * (GID_MAX_K + 1) / 2 + GID_MAX_K;   // per-channel accumulators
constexpr size_t kOffScalars = 0;
constexpr size_t kOffColors = (sizeof(DevScalars) + 255) / 256 * 256;
constexpr size_t kOffPartial = kOffColors + (sizeof(DevColors) + 255) / 256 * 256;
constexpr size_t kPartialBytes = sizeof(double) * (size_t)kMaxDenseBlocks * 3 * kMaxAcc;
constexpr size_t kNeed = kOffPartial + kPartialBytes;
static_assert(kNeed <= GID_NOALLOC_SCRATCH_BYTES, "scratch array too small for the dense reduction");

constexpr int kMaxDevices = 64;

}  // namespace

// Scratch shared by every call on a device (see the contract in gid.h).
static __device__ __align__(256) unsigned char g_noalloc_scratch[GID_NOALLOC_SCRATCH_BYTES];

static std::mutex g_mu;
static char* g_scratch_addr[kMaxDevices];  // device address of g_noalloc_scratch, per device

// Error text goes to the caller's buffer (if any): no library-side state.
struct ErrOut {
  char* buf;
  int len;
};

static int noalloc_fail(const ErrOut& eo, int code, const std::string& m) {
  if (eo.buf && eo.len > 0) {
    const size_t n = std::min((size_t)eo.len - 1, m.size());
    memcpy(eo.buf, m.data(), n);
    eo.buf[n] = '\0';
  }
  return code;
}

// One-time set-up per device: resolve the scratch array's device address with
// that device current.
static int scratch_address(const ErrOut& eo, char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(eo, GID_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(eo, GID_ERR_INVALID_ARG, "device index beyond 64");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return noalloc_fail(eo, GID_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<char*>(p);
  }
  *out = g_scratch_addr[dev];
  return GID_OK;
}

template <int K>
static void launch_dense(const Params& P, int nblk, cudaStream_t s) {
  k_dense<K, false><<<dim3(nblk, 3), 256, 0, s>>>(P, 1);
}

extern "C" int gid_dense_refine_noalloc(int H, int W, int K, const float* X_dev, const float* rgb_dev,
                                        const float* b_init_host, const gid_weights* w, void* stream,
                                        double* A_dev, double* g_dev, float* b_dev, char* errbuf,
                                        int errbuf_len) {
  const ErrOut eo{errbuf, errbuf_len};
  if (!X_dev || !rgb_dev || !b_init_host || !w) return noalloc_fail(eo, GID_ERR_INVALID_ARG, "NULL input pointer");
  if (K < 1 || K > GID_MAX_K) return noalloc_fail(eo, GID_ERR_INVALID_ARG, "K must be in 1..GID_MAX_K");
  if (H < 1 || W < 1 || (long)H * W > (1L << 28))
    return noalloc_fail(eo, GID_ERR_INVALID_ARG, "H x W must be in 1..2^28 pixels");
  const long P = (long)H * W;
  const int nblk = std::max(1, std::min(H, kMaxDenseBlocks));  // rows per block, as the context path
  const size_t need = kOffPartial + sizeof(double) * (size_t)nblk * 3 * (K * (K + 1) / 2 + K);
  if (need > GID_NOALLOC_SCRATCH_BYTES)
    return noalloc_fail(eo, GID_ERR_INVALID_ARG, "problem needs more scratch than GID_NOALLOC_SCRATCH_BYTES");
  for (int i = 0; i < 3 * K; i++)
    if (!(b_init_host[i] > 0.f) || !(b_init_host[i] < 3.4e38f))
      return noalloc_fail(eo, GID_ERR_INVALID_ARG, "initial base colours must be finite and > 0");
  char* base = nullptr;
  if (int rc = scratch_address(eo, &base)) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  DevScalars* sc = reinterpret_cast<DevScalars*>(base + kOffScalars);
  DevColors* col = reinterpret_cast<DevColors*>(base + kOffColors);
  // The completion counter and status must start at zero; the colour table holds b = b_init.
  DevColors h;
  memset(&h, 0, sizeof(h));
  for (int i = 0; i < 3 * K; i++) h.b[i] = h.binit[i] = b_init_host[i], h.bd[i] = b_init_host[i];
  cudaError_t e = cudaMemsetAsync(sc, 0, sizeof(DevScalars), s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(col, &h, sizeof(h), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return noalloc_fail(eo, GID_ERR_CUDA, std::string("scratch set-up: ") + cudaGetErrorString(e));

  Params Pm;
  memset(&Pm, 0, sizeof(Pm));
  Pm.H = H;
  Pm.W = W;
  Pm.pitch = W;  // the caller's planes are contiguous
  Pm.plane = P;
  Pm.w.ld = w->lambda_data;
  Pm.w.lIR = w->lambda_IR;
  Pm.w.lCR = w->lambda_CR;
  Pm.I = rgb_dev;
  Pm.X = const_cast<float*>(X_dev);  // read only in k_dense
  Pm.col = col;
  Pm.sc = sc;
  Pm.partial = reinterpret_cast<double*>(base + kOffPartial);
  switch (K) {
    case 1: launch_dense<1>(Pm, nblk, s); break;
    case 2: launch_dense<2>(Pm, nblk, s); break;
    case 3: launch_dense<3>(Pm, nblk, s); break;
    case 4: launch_dense<4>(Pm, nblk, s); break;
    case 5: launch_dense<5>(Pm, nblk, s); break;
    case 6: launch_dense<6>(Pm, nblk, s); break;
    case 7: launch_dense<7>(Pm, nblk, s); break;
    case 8: launch_dense<8>(Pm, nblk, s); break;
    case 9: launch_dense<9>(Pm, nblk, s); break;
    default: launch_dense<10>(Pm, nblk, s); break;
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return noalloc_fail(eo, GID_ERR_CUDA, std::string("k_dense: ") + cudaGetErrorString(e));
  if (A_dev) e = cudaMemcpyAsync(A_dev, sc->A, sizeof(double) * 3 * K * K, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && g_dev) e = cudaMemcpyAsync(g_dev, sc->g, sizeof(double) * 3 * K, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess && b_dev) e = cudaMemcpyAsync(b_dev, col->b, sizeof(float) * 3 * K, cudaMemcpyDeviceToDevice, s);
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, &sc->status, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return noalloc_fail(eo, GID_ERR_CUDA, std::string("read-back: ") + cudaGetErrorString(e));
  if (status & ST_SINGULAR) return noalloc_fail(eo, GID_ERR_NUMERIC, "base-colour normal equations not positive definite");
  return GID_OK;
}
