// Host side of the warm-start encoder-decoder: weights (FP32 masters, packed
// BF16 copies, Adam moments), the activation arena and the forward / backward
// launch sequences.  See include/gid.h for the contract of every entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/gid.h"
#include "gid_net_internal.h"
#include "gid_net_kernels.cuh"
#include "gid_nvtx.h"

using namespace gidnet;

namespace {

struct Layer {
  int ci, co, k;   // logical sizes (weights blob order: W (co, ci, k, k), bias (co))
  int cop, taps;   // output channels padded to a multiple of 32; k * k
  long w_off;      // [cop][taps][ci] in the flat fp32 masters
  long b_off;      // [cop]
  long q_off;      // offset of the layer's packed bf16 weights
};

enum { E1A, E1B, E2A, E2B, E3A, E3B, E4A, E4B, D3A, D3B, D2A, D2B, D1A, D1B, HEAD, NLAYERS };
constexpr int IN_CH = 16, HEAD_CH = 32;

// splitmix64 (Steele, Lea and Flood 2014) -> uniform doubles in (0, 1)
struct SplitMix {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
  double normal() {  // Box-Muller
    const double u = uniform(), v = uniform();
    return std::sqrt(-2.0 * std::log(u)) * std::cos(6.283185307179586 * v);
  }
};

}  // namespace

struct gid_net {
  int K = 0, wd[4] = {32, 64, 96, 128};
  Layer L[NLAYERS];
  long n_master = 0, n_packed = 0, n_params = 0;
  float *master = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  bf16 *wb = nullptr, *wt = nullptr;
  int adam_t = 0;
  float3 lw = make_float3(1.f, 1.f, 1.f);  // loss weights of r, T_0, T_1..T_K
  cudaStream_t stream = nullptr;  // the stream given at creation
  cudaStream_t s = nullptr;       // the stream of the call in progress
  // activation arena for `cap` full-resolution pixels (with gradients if cap_train)
  long cap = 0;
  bool cap_train = false;
  char* arena = nullptr;
  double* lossp = nullptr;
  std::vector<double> lossp_host;
  bf16 *x = nullptr, *a1 = nullptr, *s1 = nullptr, *da1 = nullptr, *d1 = nullptr;
  bf16 *p1 = nullptr, *a2 = nullptr, *s2 = nullptr, *da2 = nullptr, *d2 = nullptr;
  bf16 *p2 = nullptr, *a3 = nullptr, *s3 = nullptr, *da3 = nullptr, *d3 = nullptr;
  bf16 *p3 = nullptr, *a4 = nullptr, *s4 = nullptr;
  float* h = nullptr;
  bf16 *gh = nullptr, *gA1 = nullptr, *gB1 = nullptr, *gup1 = nullptr, *gs1 = nullptr;
  bf16 *gA2 = nullptr, *gB2 = nullptr, *gup2 = nullptr, *gs2 = nullptr, *gp1 = nullptr;
  bf16 *gA3 = nullptr, *gB3 = nullptr, *gup3 = nullptr, *gs3 = nullptr, *gp2 = nullptr;
  bf16 *gA4 = nullptr, *gB4 = nullptr, *gp3 = nullptr;
  int* status = nullptr;  // device word: bit 0 = a bounded wait of the tensor-core convolution gave up
  long long launches = 0;
  long long* extra_count = nullptr;  // a solver context's launch counter during gid_init_learned
  std::string err;
};

static std::string g_net_create_err;

static int nfail(gid_net* n, int code, const char* what, const char* detail = nullptr) {
  std::string m = what;
  if (detail) m += std::string(": ") + detail;
  if (n)
    n->err = m;
  else
    g_net_create_err = m;
  return code;
}

#define NET_TRY_CUDA(n, call)                                                              \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) return nfail((n), GID_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

static void counted(gid_net* n) {
  n->launches++;
  if (n->extra_count) (*n->extra_count)++;
}

static int check(gid_net* n, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return nfail(n, GID_ERR_CUDA, what, cudaGetErrorString(e));
  return GID_OK;
}

static unsigned blocks_for(long n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Reads and clears the device status word (the stream must be synchronised).
static int check_status(gid_net* n) {
  int st = 0;
  NET_TRY_CUDA(n, cudaMemcpy(&st, n->status, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    NET_TRY_CUDA(n, cudaMemset(n->status, 0, sizeof(int)));
    return nfail(n, GID_ERR_TIMEOUT, "a bounded wait of the tensor-core convolution gave up");
  }
  return GID_OK;
}

// ---------------------------------------------------------------- launches

// Pipeline depth of the tensor-core convolution for N output channels: the
// copies are the bottleneck, so the ring is kept small enough for 3-5 CTAs
// (12-20 copying warps) per SM (3 stages measured slower); TMEM (N columns
// each, rounded up to a power of two) stays within the SM's 512 columns.
static int tc_stages(int) { return 2; }
// Its dynamic shared memory: the stages of A (128 pixels x 64 bf16) and B
// (N x 64 bf16), plus 1 KB of slack for the 1024-byte alignment of the tiles.
static size_t tc_smem_bytes(int N) { return (size_t)tc_stages(N) * (TC_BM * 128 + N * 128) + 1024; }

static void conv(gid_net* n, const bf16* in1, int C1, int up1, const bf16* in2, int C2, const bf16* w,
                 const float* bias, int taps, int Co1, int Co2, bf16* out1, bf16* out2, float* out32,
                 const bf16* mask, int relu, int B, int H, int W) {
  ConvArgs a;
  a.in1 = in1;
  a.in2 = in2;
  a.C1 = C1;
  a.C2 = C2;
  a.up1 = up1;
  a.w = w;
  a.bias = bias;
  a.out1 = out1;
  a.out2 = out2;
  a.out32 = out32;
  a.mask = mask;
  a.Co1 = Co1;
  a.Co2 = Co2;
  a.B = B;
  a.H = H;
  a.W = W;
  a.taps = taps;
  a.relu = relu;
  const long P = (long)B * H * W;
  const int Co = Co1 + Co2;
  const unsigned gx = (unsigned)((P + TC_BM - 1) / TC_BM);
  k_conv_tc<2><<<gx, TC_BM, tc_smem_bytes(Co), n->s>>>(a, n->status);
  counted(n);
}

static void fwd(gid_net* n, int l, const bf16* in1, int up1, const bf16* in2, bf16* out, int B, int H, int W) {
  const Layer& L = n->L[l];
  const int C2 = in2 ? (l == D3A ? n->wd[2] : l == D2A ? n->wd[1] : n->wd[0]) : 0;
  conv(n, in1, L.ci - C2, up1, in2, C2, n->wb + L.q_off, n->master + L.b_off, L.taps, L.cop, 0, out, nullptr,
       nullptr, nullptr, 1, B, H, W);
}

// Input gradient of layer l from its pre-activation gradient g: split into
// (Co1, Co2) channels, masked by `mask` (> 0) when not split.
static void dgrad(gid_net* n, int l, const bf16* g, int Co1, bf16* out1, int Co2, bf16* out2, const bf16* mask,
                  int B, int H, int W) {
  const Layer& L = n->L[l];
  conv(n, g, L.cop, 0, nullptr, 0, n->wt + L.q_off, nullptr, L.taps, Co1, Co2, out1, out2, nullptr, mask, 0, B, H,
       W);
}

// Weight and bias gradients of layer l (accumulated into the gradient buffer).
static void wgrad(gid_net* n, int l, const bf16* g, const bf16* in1, int up1, const bf16* in2, int B, int H, int W) {
  const Layer& L = n->L[l];
  const int C2 = in2 ? (l == D3A ? n->wd[2] : l == D2A ? n->wd[1] : n->wd[0]) : 0;
  WgradArgs a;
  a.g = g;
  a.in1 = in1;
  a.in2 = in2;
  a.C1 = L.ci - C2;
  a.C2 = C2;
  a.up1 = up1;
  a.Co = L.cop;
  a.dw = n->grad + L.w_off;
  a.B = B;
  a.H = H;
  a.W = W;
  a.taps = L.taps;
  const long P = (long)B * H * W;
  // 128 output channels x WT_BN columns per CTA, the pixels split so that the
  // grid fills about two waves; each split is a whole number of 64-pixel chunks
  const int N = L.taps * L.ci;
  const unsigned gx = (L.cop + 127) / 128, gy = (N + WT_BN - 1) / WT_BN;
  const long base = (long)gx * gy;
  long splits = std::max(1L, std::min((888 + base - 1) / base, (P + WT_BK - 1) / WT_BK));
  long chunk = (P + splits - 1) / splits;
  chunk = (chunk + WT_BK - 1) / WT_BK * WT_BK;
  splits = (P + chunk - 1) / chunk;
  a.chunk = chunk;
  k_wgrad_tc<2><<<dim3(gx, gy, (unsigned)splits), 128, wgrad_tc_smem_bytes(), n->s>>>(a, n->status);
  counted(n);
  k_bias_grad<<<(unsigned)std::min(296L, std::max(1L, P / 64)), L.cop, 0, n->s>>>(g, P, L.cop, n->grad + L.b_off);
  counted(n);
}

static void pack_all(gid_net* n) {
  for (int l = 0; l < NLAYERS; l++) {
    const Layer& L = n->L[l];
    const long cnt = (long)L.cop * L.taps * L.ci;
    k_pack_weights<<<blocks_for(cnt), 256, 0, n->s>>>(n->master + L.w_off, n->wb + L.q_off, n->wt + L.q_off, L.cop,
                                                      L.taps, L.ci);
    counted(n);
  }
}

// ---------------------------------------------------------------- arena

static int ensure_arena(gid_net* n, long P1, bool train) {
  if (P1 <= n->cap && (!train || n->cap_train)) return GID_OK;
  train = train || n->cap_train;
  P1 = std::max(P1, n->cap);
  if (n->arena) {
    NET_TRY_CUDA(n, cudaDeviceSynchronize());
    cudaFree(n->arena);
    cudaFree(n->lossp);
    n->arena = nullptr;
    n->lossp = nullptr;
    n->cap = 0;
  }
  const long P2 = P1 / 4, P3 = P1 / 16, P4 = P1 / 64;
  const int w1 = n->wd[0], w2 = n->wd[1], w3 = n->wd[2], w4 = n->wd[3];
  struct Slot {
    void** dst;
    long bytes;
  };
  std::vector<Slot> slots;
  auto b16 = [&](bf16** d, long elems) { slots.push_back({(void**)d, elems * 2}); };
  b16(&n->x, P1 * IN_CH);
  b16(&n->a1, P1 * w1);
  b16(&n->s1, P1 * w1);
  b16(&n->da1, P1 * w1);
  b16(&n->d1, P1 * w1);
  b16(&n->p1, P2 * w1);
  b16(&n->a2, P2 * w2);
  b16(&n->s2, P2 * w2);
  b16(&n->da2, P2 * w2);
  b16(&n->d2, P2 * w2);
  b16(&n->p2, P3 * w2);
  b16(&n->a3, P3 * w3);
  b16(&n->s3, P3 * w3);
  b16(&n->da3, P3 * w3);
  b16(&n->d3, P3 * w3);
  b16(&n->p3, P4 * w3);
  b16(&n->a4, P4 * w4);
  b16(&n->s4, P4 * w4);
  slots.push_back({(void**)&n->h, P1 * HEAD_CH * 4});
  if (train) {
    b16(&n->gh, P1 * HEAD_CH);
    b16(&n->gA1, P1 * w1);
    b16(&n->gB1, P1 * w1);
    b16(&n->gup1, P1 * w2);
    b16(&n->gs1, P1 * w1);
    b16(&n->gA2, P2 * w2);
    b16(&n->gB2, P2 * w2);
    b16(&n->gup2, P2 * w3);
    b16(&n->gs2, P2 * w2);
    b16(&n->gp1, P2 * w1);
    b16(&n->gA3, P3 * w3);
    b16(&n->gB3, P3 * w3);
    b16(&n->gup3, P3 * w4);
    b16(&n->gs3, P3 * w3);
    b16(&n->gp2, P3 * w2);
    b16(&n->gA4, P4 * w4);
    b16(&n->gB4, P4 * w4);
    b16(&n->gp3, P4 * w3);
  }
  size_t total = 0;
  for (auto& s : slots) total += (size_t)(s.bytes + 255) / 256 * 256;
  char* base = nullptr;
  if (cudaMalloc(&base, total) != cudaSuccess) {
    cudaGetLastError();
    return nfail(n, GID_ERR_OOM, "network activation arena");
  }
  size_t o = 0;
  for (auto& s : slots) {
    *s.dst = base + o;
    o += (size_t)(s.bytes + 255) / 256 * 256;
  }
  const long nb = (P1 + 255) / 256;
  if (cudaMalloc(&n->lossp, sizeof(double) * nb) != cudaSuccess) {
    cudaGetLastError();
    cudaFree(base);
    return nfail(n, GID_ERR_OOM, "loss partials");
  }
  n->lossp_host.assign(nb, 0.0);
  n->arena = base;
  n->cap = P1;
  n->cap_train = train;
  return GID_OK;
}

// ---------------------------------------------------------------- passes

// Encoder-decoder up to the head's fp32 output h (input x already packed).
static void forward_body(gid_net* n, int B, int H, int W) {
  const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
  const int w1 = n->wd[0], w2 = n->wd[1], w3 = n->wd[2];
  fwd(n, E1A, n->x, 0, nullptr, n->a1, B, H, W);
  fwd(n, E1B, n->a1, 0, nullptr, n->s1, B, H, W);
  k_pool2<<<blocks_for((long)B * H2 * W2 * w1), 256, 0, n->s>>>(n->s1, n->p1, B, H, W, w1);
  counted(n);
  fwd(n, E2A, n->p1, 0, nullptr, n->a2, B, H2, W2);
  fwd(n, E2B, n->a2, 0, nullptr, n->s2, B, H2, W2);
  k_pool2<<<blocks_for((long)B * H4 * W4 * w2), 256, 0, n->s>>>(n->s2, n->p2, B, H2, W2, w2);
  counted(n);
  fwd(n, E3A, n->p2, 0, nullptr, n->a3, B, H4, W4);
  fwd(n, E3B, n->a3, 0, nullptr, n->s3, B, H4, W4);
  k_pool2<<<blocks_for((long)B * H8 * W8 * w3), 256, 0, n->s>>>(n->s3, n->p3, B, H4, W4, w3);
  counted(n);
  fwd(n, E4A, n->p3, 0, nullptr, n->a4, B, H8, W8);
  fwd(n, E4B, n->a4, 0, nullptr, n->s4, B, H8, W8);
  fwd(n, D3A, n->s4, 1, n->s3, n->da3, B, H4, W4);
  fwd(n, D3B, n->da3, 0, nullptr, n->d3, B, H4, W4);
  fwd(n, D2A, n->d3, 1, n->s2, n->da2, B, H2, W2);
  fwd(n, D2B, n->da2, 0, nullptr, n->d2, B, H2, W2);
  fwd(n, D1A, n->d2, 1, n->s1, n->da1, B, H, W);
  fwd(n, D1B, n->da1, 0, nullptr, n->d1, B, H, W);
  const Layer& hd = n->L[HEAD];
  conv(n, n->d1, w1, 0, nullptr, 0, n->wb + hd.q_off, n->master + hd.b_off, 1, hd.cop, 0, nullptr, nullptr, n->h,
       nullptr, 0, B, H, W);
}

// Gradients of every layer from dL/dh (in gh), accumulated into n->grad.
static void backward_body(gid_net* n, int B, int H, int W) {
  const int H2 = H / 2, W2 = W / 2, H4 = H / 4, W4 = W / 4, H8 = H / 8, W8 = W / 8;
  const int w1 = n->wd[0], w2 = n->wd[1], w3 = n->wd[2], w4 = n->wd[3];
  const Layer& hd = n->L[HEAD];
  // head (1x1, no activation)
  wgrad(n, HEAD, n->gh, n->d1, 0, nullptr, B, H, W);
  conv(n, n->gh, hd.cop, 0, nullptr, 0, n->wt + hd.q_off, nullptr, 1, w1, 0, n->gA1, nullptr, nullptr, n->d1, 0, B, H,
       W);
  // decoder level 1
  wgrad(n, D1B, n->gA1, n->da1, 0, nullptr, B, H, W);
  dgrad(n, D1B, n->gA1, w1, n->gB1, 0, nullptr, n->da1, B, H, W);
  wgrad(n, D1A, n->gB1, n->d2, 1, n->s1, B, H, W);
  dgrad(n, D1A, n->gB1, w2, n->gup1, w1, n->gs1, nullptr, B, H, W);
  k_up2_bwd<<<blocks_for((long)B * H2 * W2 * w2), 256, 0, n->s>>>(n->gup1, n->d2, n->gA2, B, H, W, w2);
  counted(n);
  // decoder level 2
  wgrad(n, D2B, n->gA2, n->da2, 0, nullptr, B, H2, W2);
  dgrad(n, D2B, n->gA2, w2, n->gB2, 0, nullptr, n->da2, B, H2, W2);
  wgrad(n, D2A, n->gB2, n->d3, 1, n->s2, B, H2, W2);
  dgrad(n, D2A, n->gB2, w3, n->gup2, w2, n->gs2, nullptr, B, H2, W2);
  k_up2_bwd<<<blocks_for((long)B * H4 * W4 * w3), 256, 0, n->s>>>(n->gup2, n->d3, n->gA3, B, H2, W2, w3);
  counted(n);
  // decoder level 3
  wgrad(n, D3B, n->gA3, n->da3, 0, nullptr, B, H4, W4);
  dgrad(n, D3B, n->gA3, w3, n->gB3, 0, nullptr, n->da3, B, H4, W4);
  wgrad(n, D3A, n->gB3, n->s4, 1, n->s3, B, H4, W4);
  dgrad(n, D3A, n->gB3, w4, n->gup3, w3, n->gs3, nullptr, B, H4, W4);
  k_up2_bwd<<<blocks_for((long)B * H8 * W8 * w4), 256, 0, n->s>>>(n->gup3, n->s4, n->gA4, B, H4, W4, w4);
  counted(n);
  // encoder level 4
  wgrad(n, E4B, n->gA4, n->a4, 0, nullptr, B, H8, W8);
  dgrad(n, E4B, n->gA4, w4, n->gB4, 0, nullptr, n->a4, B, H8, W8);
  wgrad(n, E4A, n->gB4, n->p3, 0, nullptr, B, H8, W8);
  dgrad(n, E4A, n->gB4, w3, n->gp3, 0, nullptr, nullptr, B, H8, W8);
  k_pool2_bwd<<<blocks_for((long)B * H4 * W4 * w3), 256, 0, n->s>>>(n->gp3, n->gs3, n->s3, n->gA3, B, H4, W4, w3);
  counted(n);
  // encoder level 3
  wgrad(n, E3B, n->gA3, n->a3, 0, nullptr, B, H4, W4);
  dgrad(n, E3B, n->gA3, w3, n->gB3, 0, nullptr, n->a3, B, H4, W4);
  wgrad(n, E3A, n->gB3, n->p2, 0, nullptr, B, H4, W4);
  dgrad(n, E3A, n->gB3, w2, n->gp2, 0, nullptr, nullptr, B, H4, W4);
  k_pool2_bwd<<<blocks_for((long)B * H2 * W2 * w2), 256, 0, n->s>>>(n->gp2, n->gs2, n->s2, n->gA2, B, H2, W2, w2);
  counted(n);
  // encoder level 2
  wgrad(n, E2B, n->gA2, n->a2, 0, nullptr, B, H2, W2);
  dgrad(n, E2B, n->gA2, w2, n->gB2, 0, nullptr, n->a2, B, H2, W2);
  wgrad(n, E2A, n->gB2, n->p1, 0, nullptr, B, H2, W2);
  dgrad(n, E2A, n->gB2, w1, n->gp1, 0, nullptr, nullptr, B, H2, W2);
  k_pool2_bwd<<<blocks_for((long)B * H * W * w1), 256, 0, n->s>>>(n->gp1, n->gs1, n->s1, n->gA1, B, H, W, w1);
  counted(n);
  // encoder level 1
  wgrad(n, E1B, n->gA1, n->a1, 0, nullptr, B, H, W);
  dgrad(n, E1B, n->gA1, w1, n->gB1, 0, nullptr, n->a1, B, H, W);
  wgrad(n, E1A, n->gB1, n->x, 0, nullptr, B, H, W);
}

static int check_dims(gid_net* n, int B, int H, int W) {
  if (B < 1 || H < 8 || W < 8 || H % 8 || W % 8)
    return nfail(n, GID_ERR_INVALID_ARG, "B >= 1 and H, W multiples of 8 (three 2x2 pools) are required");
  if ((long)B * H * W > (1L << 27)) return nfail(n, GID_ERR_INVALID_ARG, "batch too large");
  return GID_OK;
}

// ---------------------------------------------------------------- ABI

extern "C" int gid_net_create(int K, const int* widths, uint64_t seed, void* stream, gid_net** out) {
  if (!out) return nfail(nullptr, GID_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (K < 1 || 7 + K > IN_CH || 2 * K + 1 > HEAD_CH) return nfail(nullptr, GID_ERR_INVALID_ARG, "K must be 1..9");
  int wd[4] = {32, 64, 96, 128};
  if (widths)
    for (int i = 0; i < 4; i++) {
      if (widths[i] < 32 || widths[i] > 256 || widths[i] % 32)
        return nfail(nullptr, GID_ERR_INVALID_ARG, "widths must be multiples of 32 in [32, 256]");
      wd[i] = widths[i];
    }
  int dev_count = 0;
  cudaError_t e = cudaGetDeviceCount(&dev_count);
  if (e != cudaSuccess || dev_count < 1)
    return nfail(nullptr, GID_ERR_CUDA, "no CUDA device", e != cudaSuccess ? cudaGetErrorString(e) : nullptr);
  gid_net* n = new (std::nothrow) gid_net();
  if (!n) return nfail(nullptr, GID_ERR_OOM, "host allocation");
  n->K = K;
  memcpy(n->wd, wd, sizeof(wd));
  n->stream = n->s = (cudaStream_t)stream;
  const int w1 = wd[0], w2 = wd[1], w3 = wd[2], w4 = wd[3];
  const int spec[NLAYERS][3] = {{IN_CH, w1, 3}, {w1, w1, 3},      {w1, w2, 3},      {w2, w2, 3}, {w2, w3, 3},
                                {w3, w3, 3},    {w3, w4, 3},      {w4, w4, 3},      {w4 + w3, w3, 3}, {w3, w3, 3},
                                {w3 + w2, w2, 3}, {w2, w2, 3},    {w2 + w1, w1, 3}, {w1, w1, 3}, {w1, 2 * K + 1, 1}};
  long off = 0, q = 0, np = 0;
  for (int l = 0; l < NLAYERS; l++) {
    Layer& L = n->L[l];
    L.ci = spec[l][0];
    L.co = spec[l][1];
    L.k = spec[l][2];
    L.taps = L.k * L.k;
    L.cop = (L.co + 31) / 32 * 32;
    L.w_off = off;
    off += (long)L.cop * L.taps * L.ci;
    L.b_off = off;
    off += L.cop;
    off = (off + 3) / 4 * 4;  // 16-byte aligned layers
    L.q_off = q;
    q += ((long)L.cop * L.taps * L.ci + 7) / 8 * 8;
    np += (long)L.co * L.ci * L.taps + L.co;
  }
  n->n_master = off;
  n->n_packed = q;
  n->n_params = np;
  auto bad = [&](const char* what) {
    gid_net_destroy(n);
    return nfail(nullptr, GID_ERR_OOM, what);
  };
  if (cudaMalloc(&n->master, 4 * sizeof(float) * off) != cudaSuccess) return bad("network weights");
  n->grad = n->master + off;
  n->m = n->grad + off;
  n->v = n->m + off;
  if (cudaMalloc(&n->wb, 2 * sizeof(bf16) * q) != cudaSuccess) return bad("packed weights");
  if (cudaMalloc(&n->status, sizeof(int)) != cudaSuccess || cudaMemset(n->status, 0, sizeof(int)) != cudaSuccess)
    return bad("status word");
  if (cudaFuncSetAttribute(k_conv_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc_smem_bytes(256)) !=
      cudaSuccess) {
    cudaGetLastError();
    gid_net_destroy(n);
    return nfail(nullptr, GID_ERR_CUDA, "tensor-core convolution: shared memory attribute");
  }
  if (cudaFuncSetAttribute(k_wgrad_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wgrad_tc_smem_bytes()) !=
      cudaSuccess) {
    cudaGetLastError();
    gid_net_destroy(n);
    return nfail(nullptr, GID_ERR_CUDA, "tensor-core weight gradient: shared memory attribute");
  }
  n->wt = n->wb + q;
  // He-normal weights, zero biases, from the seed
  std::vector<float> h(off, 0.f);
  SplitMix rng{seed};
  for (int l = 0; l < NLAYERS; l++) {
    const Layer& L = n->L[l];
    const double sd = std::sqrt(2.0 / (L.ci * L.taps));
    for (int o = 0; o < L.co; o++)
      for (long j = 0; j < (long)L.taps * L.ci; j++) h[L.w_off + (long)o * L.taps * L.ci + j] = (float)(sd * rng.normal());
  }
  if (cudaMemcpy(n->master, h.data(), sizeof(float) * off, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(n->grad, 0, 3 * sizeof(float) * off) != cudaSuccess)
    return bad("weight upload");
  pack_all(n);
  if (cudaStreamSynchronize(n->s) != cudaSuccess) return bad("weight packing");
  *out = n;
  return GID_OK;
}

extern "C" void gid_net_destroy(gid_net* n) {
  if (!n) return;
  if (n->s) cudaStreamSynchronize(n->s);
  cudaFree(n->master);
  cudaFree(n->wb);
  cudaFree(n->arena);
  cudaFree(n->lossp);
  cudaFree(n->status);
  delete n;
}

extern "C" const char* gid_net_last_error(const gid_net* n) { return n ? n->err.c_str() : g_net_create_err.c_str(); }

extern "C" long gid_net_num_params(const gid_net* n) { return n ? n->n_params : 0; }

extern "C" long long gid_net_launch_count(const gid_net* n) { return n ? n->launches : 0; }

// blob (per layer W (co, ci, k, k) then b (co)) <-> internal [cop][taps][ci] + [cop]
static void blob_to_internal(const gid_net* n, const float* blob, float* h) {
  long o = 0;
  for (int l = 0; l < NLAYERS; l++) {
    const Layer& L = n->L[l];
    for (int co = 0; co < L.co; co++)
      for (int ci = 0; ci < L.ci; ci++)
        for (int t = 0; t < L.taps; t++) h[L.w_off + ((long)co * L.taps + t) * L.ci + ci] = blob[o++];
    for (int co = 0; co < L.co; co++) h[L.b_off + co] = blob[o++];
  }
}
static void internal_to_blob(const gid_net* n, const float* h, float* blob) {
  long o = 0;
  for (int l = 0; l < NLAYERS; l++) {
    const Layer& L = n->L[l];
    for (int co = 0; co < L.co; co++)
      for (int ci = 0; ci < L.ci; ci++)
        for (int t = 0; t < L.taps; t++) blob[o++] = h[L.w_off + ((long)co * L.taps + t) * L.ci + ci];
    for (int co = 0; co < L.co; co++) blob[o++] = h[L.b_off + co];
  }
}

extern "C" int gid_net_set_weights(gid_net* n, const float* blob_host) {
  if (!n || !blob_host) return nfail(n, GID_ERR_INVALID_ARG, "NULL argument");
  for (long i = 0; i < n->n_params; i++)
    if (!std::isfinite(blob_host[i])) return nfail(n, GID_ERR_INVALID_ARG, "weights must be finite");
  std::vector<float> h(n->n_master, 0.f);
  blob_to_internal(n, blob_host, h.data());
  n->s = n->stream;
  NET_TRY_CUDA(n, cudaMemcpyAsync(n->master, h.data(), sizeof(float) * n->n_master, cudaMemcpyHostToDevice, n->s));
  NET_TRY_CUDA(n, cudaMemsetAsync(n->m, 0, 2 * sizeof(float) * n->n_master, n->s));
  n->adam_t = 0;
  pack_all(n);
  if (int rc = check(n, "k_pack_weights")) return rc;
  NET_TRY_CUDA(n, cudaStreamSynchronize(n->s));
  return GID_OK;
}

static int get_blob(gid_net* n, const float* dev, float* blob_host) {
  if (!n || !blob_host) return nfail(n, GID_ERR_INVALID_ARG, "NULL argument");
  std::vector<float> h(n->n_master);
  n->s = n->stream;
  NET_TRY_CUDA(n, cudaMemcpyAsync(h.data(), dev, sizeof(float) * n->n_master, cudaMemcpyDeviceToHost, n->s));
  NET_TRY_CUDA(n, cudaStreamSynchronize(n->s));
  internal_to_blob(n, h.data(), blob_host);
  return check_status(n);
}

extern "C" int gid_net_get_weights(gid_net* n, float* blob_host) { return get_blob(n, n ? n->master : nullptr, blob_host); }

extern "C" int gid_net_get_grads(gid_net* n, float* blob_host) { return get_blob(n, n ? n->grad : nullptr, blob_host); }

static void pack_input(gid_net* n, const float* rgb, Planes rg, const uint8_t* lab, long lab_bs, long lab_rs,
                       const float* palette, int B, int H, int W) {
  const long P = (long)B * H * W;
  k_pack_input<<<blocks_for(P), 256, 0, n->s>>>(rgb, rg, lab, lab_bs, lab_rs, palette, n->K, B, H, W, n->x);
  counted(n);
}

extern "C" int gid_net_forward(gid_net* n, int B, int H, int W, const float* rgb_dev, const uint8_t* labels_dev,
                               const float* palette_dev, float* r_dev, float* T_dev) {
  gid::NvtxRange nvtx_range("gid_net_forward");
  if (!n || !rgb_dev || !labels_dev || !palette_dev) return nfail(n, GID_ERR_INVALID_ARG, "NULL argument");
  if (int rc = check_dims(n, B, H, W)) return rc;
  n->s = n->stream;
  const long HW = (long)H * W, P = (long)B * HW;
  if (int rc = ensure_arena(n, P, false)) return rc;
  pack_input(n, rgb_dev, Planes{3 * HW, HW, W}, labels_dev, HW, W, palette_dev, B, H, W);
  forward_body(n, B, H, W);
  k_head<<<blocks_for(P), 256, 0, n->s>>>(n->h, HEAD_CH, palette_dev, n->K, B, H, W, r_dev, Planes{3 * HW, HW, W},
                                           T_dev, Planes{(n->K + 1) * HW, HW, W}, nullptr, nullptr, nullptr, nullptr, n->lw,
                                           0.f);
  counted(n);
  return check(n, "network forward");
}

extern "C" int gid_net_backward(gid_net* n, int B, int H, int W, const float* rgb_dev, const uint8_t* labels_dev,
                                const float* palette_dev, const float* r_target_dev, const float* T_target_dev,
                                double* loss_host) {
  gid::NvtxRange nvtx_range("gid_net_backward");
  if (!n || !rgb_dev || !labels_dev || !palette_dev || !r_target_dev || !T_target_dev)
    return nfail(n, GID_ERR_INVALID_ARG, "NULL argument");
  if (int rc = check_dims(n, B, H, W)) return rc;
  n->s = n->stream;
  const long HW = (long)H * W, P = (long)B * HW;
  if (int rc = ensure_arena(n, P, true)) return rc;
  NET_TRY_CUDA(n, cudaMemsetAsync(n->grad, 0, sizeof(float) * n->n_master, n->s));
  pack_input(n, rgb_dev, Planes{3 * HW, HW, W}, labels_dev, HW, W, palette_dev, B, H, W);
  forward_body(n, B, H, W);
  const unsigned nb = blocks_for(P);
  k_head<<<nb, 256, 0, n->s>>>(n->h, HEAD_CH, palette_dev, n->K, B, H, W, nullptr, Planes{0, 0, 0}, nullptr,
                               Planes{0, 0, 0}, r_target_dev, T_target_dev, n->gh, n->lossp, n->lw, 0.f);
  counted(n);
  backward_body(n, B, H, W);
  if (int rc = check(n, "network backward")) return rc;
  if (loss_host) {
    NET_TRY_CUDA(n, cudaMemcpyAsync(n->lossp_host.data(), n->lossp, sizeof(double) * nb, cudaMemcpyDeviceToHost, n->s));
    NET_TRY_CUDA(n, cudaStreamSynchronize(n->s));
    if (int rc = check_status(n)) return rc;
    double t = 0.0;
    for (unsigned i = 0; i < nb; i++) t += n->lossp_host[i];
    *loss_host = t;
    if (!std::isfinite(t)) return nfail(n, GID_ERR_NUMERIC, "loss is not finite");
  }
  return GID_OK;
}

extern "C" int gid_net_set_loss_weights(gid_net* n, float w_r, float w_T0, float w_Tk) {
  if (!n) return nfail(n, GID_ERR_INVALID_ARG, "NULL net");
  if (!(w_r >= 0.f) || !(w_T0 >= 0.f) || !(w_Tk >= 0.f) || !std::isfinite(w_r + w_T0 + w_Tk))
    return nfail(n, GID_ERR_INVALID_ARG, "loss weights must be finite and >= 0");
  n->lw = make_float3(w_r, w_T0, w_Tk);
  return GID_OK;
}

extern "C" int gid_net_adam_step(gid_net* n, float lr, float beta1, float beta2, float eps) {
  if (!n) return nfail(n, GID_ERR_INVALID_ARG, "NULL net");
  if (!(lr >= 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps >= 0.f))
    return nfail(n, GID_ERR_INVALID_ARG, "bad Adam hyper-parameters");
  n->s = n->stream;
  n->adam_t++;
  const float c1 = 1.f - (float)std::pow((double)beta1, n->adam_t), c2 = 1.f - (float)std::pow((double)beta2, n->adam_t);
  k_adam<<<blocks_for(n->n_master), 256, 0, n->s>>>(n->master, n->grad, n->m, n->v, n->n_master, lr, beta1, beta2, eps,
                                                    c1, c2);
  counted(n);
  pack_all(n);
  return check(n, "k_adam");
}

// ---------------------------------------------------------------- solver init

int gidnet_K(const gid_net* n) { return n->K; }

int gidnet_infer_planes(gid_net* n, int H, int W, const float* I, long plane, int pitch, const uint8_t* lab,
                        const float* palette, float tk_zero, float* X, cudaStream_t s, long long* launches,
                        std::string* err) {
  n->s = s;
  n->extra_count = launches;
  int rc = check_dims(n, 1, H, W);
  if (!rc) rc = ensure_arena(n, (long)H * W, false);
  if (!rc) {
    pack_input(n, I, Planes{0, plane, pitch}, lab, 0, pitch, palette, 1, H, W);
    forward_body(n, 1, H, W);
    k_head<<<blocks_for((long)H * W), 256, 0, n->s>>>(n->h, HEAD_CH, palette, n->K, 1, H, W, X, Planes{0, plane, pitch},
                                                       X + 3 * plane, Planes{0, plane, pitch}, nullptr, nullptr, nullptr,
                                                       nullptr, n->lw, tk_zero);
    counted(n);
    rc = check(n, "network forward (learned initial state)");
  }
  n->extra_count = nullptr;
  n->s = n->stream;
  if (rc && err) *err = n->err;
  return rc;
}
