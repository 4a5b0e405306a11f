// Kernels of the warm-start encoder-decoder (BF16 tensor cores, FP32 accumulate).
//
// Activations are NHWC bfloat16, pixel-major (p = (b H + y) W + x) with the
// channel count a multiple of 16.  Weights are [C_out][tap][C_in] bfloat16
// (taps = 9 for 3x3, 1 for 1x1), packed from FP32 master weights.
//
// A convolution is an implicit GEMM, M = pixels, N = output channels,
// K = taps x input channels, on the 5th-generation tensor cores (tcgen05.mma,
// bf16 operands in shared memory, fp32 accumulator in tensor memory; k_conv_tc
// below).  The input may be the channel concatenation of two tensors (the
// decoder's skip connections), the first of them read through a nearest 2x
// upsampling (so the upsampled tensor is never stored); the output may be split
// into two tensors (the gradient of such a concatenation).  The input gradient
// is the same kernel on the output gradient with the weights flipped in space
// and transposed in channels.  The weight gradient is a GEMM over pixels
// (M = output channels, N = taps x input channels) split across blocks, also
// on the tensor cores (operands staged MN-major from the NHWC tensors), reduced
// with FP32 atomics.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gidnet {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte asynchronous global -> shared copy; src_bytes = 0 writes zeros.
__device__ __forceinline__ void cp16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
  const bf16 a = __float2bfloat16(lo), b = __float2bfloat16(hi);
  return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

__device__ __forceinline__ float bf(bf16 v) { return __bfloat162float(v); }

// Pixel coordinates of a flat NHWC pixel index.
struct Pix {
  int b, y, x;
};
__device__ __forceinline__ Pix pix_of(long p, int H, int W) {
  Pix r;
  r.x = (int)(p % W);
  const long q = p / W;
  r.y = (int)(q % H);
  r.b = (int)(q / H);
  return r;
}

// Address (in elements) of channel `c` of pixel (b, yy, xx) of a tensor with
// `cs` channels stored at full (up = 0) or half (up = 1) resolution.
__device__ __forceinline__ long tensor_off(int b, int yy, int xx, int H, int W, int up, int cs, int c) {
  const long pix = up ? ((long)b * (H >> 1) + (yy >> 1)) * (W >> 1) + (xx >> 1) : ((long)b * H + yy) * W + xx;
  return pix * cs + c;
}

struct ConvArgs {
  const bf16* in1;  // NHWC, C1 channels; half resolution if up1
  const bf16* in2;  // NHWC, C2 channels (input channels C1..), or NULL if C2 == 0
  int C1, C2, up1;
  const bf16* w;      // [Co1 + Co2][taps][C1 + C2]
  const float* bias;  // [Co1 + Co2] or NULL
  bf16* out1;         // NHWC, Co1 channels (output channels 0..Co1-1)
  bf16* out2;         // NHWC, Co2 channels (output channels Co1..), or NULL
  float* out32;       // fp32 NHWC (Co1 + Co2 channels) instead of out1/out2, or NULL
  const bf16* mask;   // if set (Co2 == 0): out1 *= (mask > 0), same shape as out1
  int Co1, Co2;
  int B, H, W, taps, relu;
};

// ---------------------------------------------------------------- tcgen05 convolution
//
// The same implicit GEMM on the 5th-generation tensor cores: D[128 pixels][N =
// all output channels] accumulates in tensor memory (FP32, one TMEM lane per
// pixel, one column per channel); K = taps x C_in flattened as k = tap C_in +
// c, in chunks of 64 (one 128-byte swizzle atom of bf16).  All 128 threads
// stage the im2col rows of A and the weight rows of B with 16-byte cp.async
// copies into K-major, 128-byte-swizzled shared tiles (a STAGES-deep ring); one
// thread issues tcgen05.mma kind::f16 (A and B bf16, D fp32, M = 128, K = 16
// per instruction) and commits each stage to an mbarrier that frees it for the
// next copies.  Waits are bounded (status bit on timeout); TMEM is allocated
// by warp 0 (at most 256 columns; at most two CTAs fit on an SM) and always
// freed before the CTA exits.

constexpr int TC_BM = 128, TC_BK = 64;
constexpr long TC_SPINS = 1L << 22;

__device__ __forceinline__ void tc_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* bar, unsigned parity) {
  for (long i = 0; i < TC_SPINS; i++) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, rows of
// 128 bytes, 8-row groups 1024 bytes apart (stride byte offset); the leading
// byte offset is not used by this layout; descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t tc_desc_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor, kind::f16: D fp32, A and B bf16, both K-major, M x N.
__host__ __device__ constexpr uint32_t tc_idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

template <int STAGES>
__global__ void __launch_bounds__(128, 1) k_conv_tc(ConvArgs a, int* __restrict__ status) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_stage[STAGES];
  __shared__ __align__(8) uint64_t bar_done;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int N = a.Co1 + a.Co2;  // 32..256, a multiple of 32
  const int Ci = a.C1 + a.C2, Ktot = a.taps * Ci, nk = (Ktot + TC_BK - 1) / TC_BK;
  const uint32_t ncols = N <= 32 ? 32u : N <= 64 ? 64u : N <= 128 ? 128u : 256u;
  const int a_bytes = TC_BM * 128, stage_bytes = a_bytes + N * 128;  // N * 128 is a multiple of 1024
  // 1024-byte aligned ring of stages (the dynamic allocation has 1 KB of slack)
  const uint32_t raw = smem_u32(tc_smem_raw);
  uint8_t* st = tc_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t st_addr = smem_u32(st);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < STAGES; i++) tc_mbar_init(&bar_stage[i]);
    tc_mbar_init(&bar_done);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  const long P = (long)a.B * a.H * a.W, p = (long)blockIdx.x * TC_BM + tid;
  const bool prow = p < P;
  const Pix px = pix_of(prow ? p : 0, a.H, a.W);

  // stage s <- K-chunk kc: A row `tid` (8 chunks of 8 channels), B rows of the weights
  auto load_stage = [&](int kc, int s) {
    uint8_t* sa = st + s * stage_bytes;
    uint8_t* sb = sa + a_bytes;
    // k = tap C_in + ch for the 8 chunks: one division, then wrap-arounds
    int tap = (kc * TC_BK) / Ci, ch = kc * TC_BK - tap * Ci;
#pragma unroll
    for (int c = 0; c < 8; c++, ch += 8) {
      while (ch >= Ci) {
        ch -= Ci;
        tap++;
      }
      const int k = kc * TC_BK + c * 8;
      const bf16* src = a.in1;
      int bytes = 0;
      if (prow && k < Ktot) {
        const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
        const int yy = px.y + dy, xx = px.x + dx;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          src = ch < a.C1 ? a.in1 + tensor_off(px.b, yy, xx, a.H, a.W, a.up1, a.C1, ch)
                          : a.in2 + tensor_off(px.b, yy, xx, a.H, a.W, 0, a.C2, ch - a.C1);
          bytes = 16;
        }
      }
      cp16(sa + tid * 128 + ((c ^ (tid & 7)) << 4), src, bytes);
    }
    for (int i = tid; i < N * 8; i += TC_BM) {
      const int r = i >> 3, c = i & 7, k = kc * TC_BK + c * 8;
      const bool ok = k < Ktot;
      cp16(sb + r * 128 + ((c ^ (r & 7)) << 4), ok ? a.w + (long)r * Ktot + k : a.w, ok ? 16 : 0);
    }
  };

  const uint32_t idesc = tc_idesc_bf16(TC_BM, N);
  bool waits_ok = true;
#pragma unroll
  for (int s = 0; s < STAGES - 1; s++) {
    if (s < nk) load_stage(s, s);
    cp_commit();
  }
  for (int kc = 0; kc < nk; kc++) {
    const int s = kc % STAGES;
    cp_wait<STAGES - 2>();  // this thread's copies of chunk kc have landed
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // ... and are visible to the tensor core
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = st_addr + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; kk++) {
        const uint64_t ad = tc_desc_sw128(sa + kk * 32), bd = tc_desc_sw128(sb + kk * 32);
        const uint32_t acc = (kc | kk) != 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&bar_stage[s]))
                   : "memory");
    }
    // chunk kc + STAGES - 1 refills the stage of chunk kc - 1 once its MMAs are done
    const int nxt = kc + STAGES - 1;
    if (nxt < nk) {
      const int ns = nxt % STAGES;
      if (kc >= 1) waits_ok &= tc_mbar_wait(&bar_stage[ns], (unsigned)(((kc - 1) / STAGES) & 1));
      load_stage(nxt, ns);
    }
    cp_commit();
  }
  if (tid == 0)
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                     smem_u32(&bar_done))
                 : "memory");
  waits_ok &= tc_mbar_wait(&bar_done, 0u);
  tc_fence_after();

  // epilogue: this thread's pixel is TMEM lane tid (warp w reads lanes 32 w ..)
  const int Co = N;
  for (int j = 0; j < N; j += 16) {
    uint32_t r[16];
    const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j;
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
    if (!prow) continue;
    float v[16];
#pragma unroll
    for (int e = 0; e < 16; e++) {
      v[e] = __uint_as_float(r[e]) + (a.bias ? a.bias[j + e] : 0.f);
      if (a.relu) v[e] = fmaxf(v[e], 0.f);
    }
    if (a.out32) {
      float4* dst = reinterpret_cast<float4*>(a.out32 + p * Co + j);
#pragma unroll
      for (int e = 0; e < 4; e++) dst[e] = make_float4(v[4 * e], v[4 * e + 1], v[4 * e + 2], v[4 * e + 3]);
      continue;
    }
    const bool first = j < a.Co1;
    if (first && a.mask) {
      const uint4* mk = reinterpret_cast<const uint4*>(a.mask + p * a.Co1 + j);
      const uint4 m0 = mk[0], m1 = mk[1];
      const uint32_t mw[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
      for (int e = 0; e < 8; e++) {
        const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw[e]);
        if (!(bf(m2.x) > 0.f)) v[2 * e] = 0.f;
        if (!(bf(m2.y) > 0.f)) v[2 * e + 1] = 0.f;
      }
    }
    uint4* dst = first ? reinterpret_cast<uint4*>(a.out1 + p * a.Co1 + j)
                       : reinterpret_cast<uint4*>(a.out2 + p * a.Co2 + (j - a.Co1));
    dst[0] = make_uint4(pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]), pack2(v[6], v[7]));
    dst[1] = make_uint4(pack2(v[8], v[9]), pack2(v[10], v[11]), pack2(v[12], v[13]), pack2(v[14], v[15]));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(ncols) : "memory");
  if (!waits_ok) atomicOr(status, 1);
}

struct WgradArgs {
  const bf16* g;    // NHWC, Co channels: dL/d(conv output before the activation)
  const bf16* in1;  // the conv's input, as in ConvArgs
  const bf16* in2;
  int C1, C2, up1;
  int Co;
  float* dw;  // [Co][taps][C1 + C2] fp32, accumulated
  int B, H, W, taps;
  long chunk;  // pixels per block along grid.z (a multiple of 64)
};

// ---------------------------------------------------------------- tcgen05 weight gradient
//
// dW[co][n] += sum_p g[p][co] in[p + offset(tap)][ci], n = tap C_in + ci, as
// D[M = co][N = n] = A[M][K] B[N][K]^T with K = pixels, on the 5th-generation
// tensor cores.  Both operands come from NHWC tensors, whose channels are
// contiguous, so both are staged MN-major: within a stage, pixel r (a K index)
// of 64-channel block j is one 128-byte row at j * 8 KB + r * 128, its 16-byte
// chunks swizzled by the row (chunk c at ((c ^ (r & 7)) << 4)), 8-row groups
// 1 KB apart along K.  One CTA: 128 output channels x WT_BN columns n in tensor
// memory, the pixels of its split in chunks of 64 (a two-stage ring of
// cp.async copies, one thread issuing tcgen05.mma), then FP32 atomics into dW.
// Waits are bounded; TMEM is always freed.
constexpr int WT_BN = 128, WT_BK = 64;

// Shared-memory descriptor, MN-major operand, 128-byte swizzle: 64-element
// blocks along M (or N) 8 KB apart (leading byte offset), 8-row groups along K
// 1 KB apart (stride byte offset), descriptor version 1.
__device__ __forceinline__ uint64_t tc_desc_mn_sw128(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(8192 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}

template <int STAGES>
__global__ void __launch_bounds__(128, 1) k_wgrad_tc(WgradArgs a, int* __restrict__ status) {
  extern __shared__ uint8_t tc_smem_raw[];
  __shared__ __align__(8) uint64_t bar_stage[STAGES];
  __shared__ __align__(8) uint64_t bar_done;
  __shared__ uint32_t tmem_slot;
  constexpr int A_BYTES = 2 * 64 * 128, B_BYTES = (WT_BN / 64) * 64 * 128, STAGE_BYTES = A_BYTES + B_BYTES;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int Ci = a.C1 + a.C2, Ntot = a.taps * Ci;
  const int m0 = blockIdx.x * 128, n0 = blockIdx.y * WT_BN;
  const long P = (long)a.B * a.H * a.W, p0 = (long)blockIdx.z * a.chunk;
  const long pend = p0 + a.chunk < P ? p0 + a.chunk : P;
  const int nk = pend > p0 ? (int)((pend - p0 + WT_BK - 1) / WT_BK) : 0;
  const uint32_t raw = smem_u32(tc_smem_raw);
  uint8_t* st = tc_smem_raw + (((raw + 1023u) & ~1023u) - raw);
  const uint32_t st_addr = smem_u32(st);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&tmem_slot)),
                 "r"((uint32_t)WT_BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < STAGES; i++) tc_mbar_init(&bar_stage[i]);
    tc_mbar_init(&bar_done);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  // stage s <- pixels p0 + 64 kc ..: A rows from g, B rows from the shifted input
  auto load_stage = [&](int kc, int s) {
    uint8_t* sa = st + s * STAGE_BYTES;
    uint8_t* sb = sa + A_BYTES;
    const long pk = p0 + (long)kc * WT_BK;
    for (int i = tid; i < 2 * 64 * 8; i += 128) {
      const int j = i >> 9, r = (i >> 3) & 63, c = i & 7;
      const long p = pk + r;
      const int co = m0 + j * 64 + c * 8;
      const bool ok = p < pend && co < a.Co;
      cp16(sa + j * 8192 + r * 128 + ((c ^ (r & 7)) << 4), ok ? a.g + p * a.Co + co : a.g, ok ? 16 : 0);
    }
    for (int i = tid; i < (WT_BN / 64) * 64 * 8; i += 128) {
      const int j = i >> 9, r = (i >> 3) & 63, c = i & 7;
      const long p = pk + r;
      const int n = n0 + j * 64 + c * 8;
      const bf16* src = a.in1;
      int bytes = 0;
      if (p < pend && n < Ntot) {
        const int tap = n / Ci, ch = n - tap * Ci;
        const Pix px = pix_of(p, a.H, a.W);
        const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
        const int yy = px.y + dy, xx = px.x + dx;
        if (yy >= 0 && yy < a.H && xx >= 0 && xx < a.W) {
          src = ch < a.C1 ? a.in1 + tensor_off(px.b, yy, xx, a.H, a.W, a.up1, a.C1, ch)
                          : a.in2 + tensor_off(px.b, yy, xx, a.H, a.W, 0, a.C2, ch - a.C1);
          bytes = 16;
        }
      }
      cp16(sb + j * 8192 + r * 128 + ((c ^ (r & 7)) << 4), src, bytes);
    }
  };

  // both operands MN-major (instruction-descriptor bits 15 and 16)
  const uint32_t idesc = tc_idesc_bf16(128, WT_BN) | (1u << 15) | (1u << 16);
  bool waits_ok = true;
#pragma unroll
  for (int s = 0; s < STAGES - 1; s++) {
    if (s < nk) load_stage(s, s);
    cp_commit();
  }
  for (int kc = 0; kc < nk; kc++) {
    const int s = kc % STAGES;
    cp_wait<STAGES - 2>();
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t sa = st_addr + s * STAGE_BYTES, sb = sa + A_BYTES;
#pragma unroll
      for (int kk = 0; kk < WT_BK / 16; kk++) {  // 16 pixels = two 8-row groups per instruction
        const uint64_t ad = tc_desc_mn_sw128(sa + kk * 2048), bd = tc_desc_mn_sw128(sb + kk * 2048);
        const uint32_t acc = (kc | kk) != 0 ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&bar_stage[s]))
                   : "memory");
    }
    const int nxt = kc + STAGES - 1;
    if (nxt < nk) {
      const int ns = nxt % STAGES;
      if (kc >= 1) waits_ok &= tc_mbar_wait(&bar_stage[ns], (unsigned)(((kc - 1) / STAGES) & 1));
      load_stage(nxt, ns);
    }
    cp_commit();
  }
  if (nk > 0) {
    if (tid == 0)
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                       smem_u32(&bar_done))
                   : "memory");
    waits_ok &= tc_mbar_wait(&bar_done, 0u);
    tc_fence_after();
    // epilogue: TMEM lane 32 w + lane is output channel m0 + 32 w + lane
    const int co = m0 + warp * 32 + (tid & 31);
    for (int j = 0; j < WT_BN; j += 16) {
      uint32_t r[16];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
      if (co >= a.Co) continue;
      float* row = a.dw + (long)co * Ntot + n0 + j;
#pragma unroll
      for (int e = 0; e < 16; e += 4)
        if (n0 + j + e < Ntot)
          atomicAdd(reinterpret_cast<float4*>(row + e), make_float4(__uint_as_float(r[e]), __uint_as_float(r[e + 1]),
                                                                   __uint_as_float(r[e + 2]), __uint_as_float(r[e + 3])));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)WT_BN) : "memory");
  if (!waits_ok) atomicOr(status, 1);
}

constexpr size_t wgrad_tc_smem_bytes() { return 2 * (2 * 64 * 128 + (WT_BN / 64) * 64 * 128) + 1024; }

// db[c] += sum_p g[p][c]; blockDim.x == C.
__global__ void k_bias_grad(const bf16* __restrict__ g, long P, int C, float* __restrict__ db) {
  const int c = threadIdx.x;
  const long per = (P + gridDim.x - 1) / gridDim.x, p0 = (long)blockIdx.x * per;
  const long p1 = p0 + per < P ? p0 + per : P;
  float s = 0.f;
  for (long p = p0; p < p1; p++) s += bf(g[p * C + c]);
  atomicAdd(db + c, s);
}

// 2 x 2 average pool, NHWC, full resolution H x W (even) -> H/2 x W/2.
__global__ void k_pool2(const bf16* __restrict__ in, bf16* __restrict__ out, int B, int H, int W, int C) {
  const long n = (long)B * (H / 2) * (W / 2) * C;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % C);
  const Pix q = pix_of(i / C, H / 2, W / 2);
  const long base = (((long)q.b * H + 2 * q.y) * W + 2 * q.x) * C + c, row = (long)W * C;
  const float s = bf(in[base]) + bf(in[base + C]) + bf(in[base + row]) + bf(in[base + row + C]);
  out[i] = __float2bfloat16(0.25f * s);
}

// gin = (pool2^T gout + add) * (mask > 0), at full resolution H x W.
__global__ void k_pool2_bwd(const bf16* __restrict__ gout, const bf16* __restrict__ add,
                            const bf16* __restrict__ mask, bf16* __restrict__ gin, int B, int H, int W, int C) {
  const long n = (long)B * H * W * C;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % C);
  const Pix q = pix_of(i / C, H, W);
  float v = 0.25f * bf(gout[(((long)q.b * (H / 2) + q.y / 2) * (W / 2) + q.x / 2) * C + c]);
  if (add) v += bf(add[i]);
  if (mask && !(bf(mask[i]) > 0.f)) v = 0.f;
  gin[i] = __float2bfloat16(v);
}

// gin = (up2^T gout) * (mask > 0): the sum of each half-resolution pixel's four
// children; gout is at full resolution H x W, gin and mask at H/2 x W/2.
__global__ void k_up2_bwd(const bf16* __restrict__ gout, const bf16* __restrict__ mask, bf16* __restrict__ gin,
                          int B, int H, int W, int C) {
  const long n = (long)B * (H / 2) * (W / 2) * C;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = (int)(i % C);
  const Pix q = pix_of(i / C, H / 2, W / 2);
  const long base = (((long)q.b * H + 2 * q.y) * W + 2 * q.x) * C + c, row = (long)W * C;
  float v = bf(gout[base]) + bf(gout[base + C]) + bf(gout[base + row]) + bf(gout[base + row + C]);
  if (mask && !(bf(mask[i]) > 0.f)) v = 0.f;
  gin[i] = __float2bfloat16(v);
}

// Planar fp32 image geometry: element (b, c, y, x) at b * bs + c * cs + y * rs + x.
struct Planes {
  long bs, cs, rs;
};

// Network input (NHWC bf16, 16 channels): the image in channels 0..2, the
// clustered reflectance palette[label] in channels 3..5, the cold-start
// shading estimate mean_c I / mean_c R_cluster in channel 6 and the one-hot
// label in channels 7..7+K-1 (K <= 9), zeros elsewhere.  Labels >= K count as 0.
__global__ void k_pack_input(const float* __restrict__ rgb, Planes rg, const uint8_t* __restrict__ lab, long lab_bs,
                             long lab_rs, const float* __restrict__ palette, int K, int B, int H, int W,
                             bf16* __restrict__ x) {
  const long P = (long)B * H * W;
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const Pix q = pix_of(p, H, W);
  int l = lab[q.b * lab_bs + (long)q.y * lab_rs + q.x];
  l = l < K ? l : 0;
  float v[6];
  for (int c = 0; c < 3; c++) {
    v[c] = rgb[q.b * rg.bs + c * rg.cs + (long)q.y * rg.rs + q.x];
    v[3 + c] = palette[(long)q.b * K * 3 + l * 3 + c];
  }
  float o[16];
  for (int c = 0; c < 6; c++) o[c] = v[c];
  o[6] = (v[0] + v[1] + v[2]) / (v[3] + v[4] + v[5]);
  for (int c = 7; c < 16; c++) o[c] = (c - 7 == l) ? 1.f : 0.f;
  uint4* dst = reinterpret_cast<uint4*>(x + p * 16);
  dst[0] = make_uint4(pack2(o[0], o[1]), pack2(o[2], o[3]), pack2(o[4], o[5]), pack2(o[6], o[7]));
  dst[1] = make_uint4(pack2(o[8], o[9]), pack2(o[10], o[11]), pack2(o[12], o[13]), pack2(o[14], o[15]));
}

// Head: h (fp32 NHWC, Ch channels: K logits w, then T_0..T_K) and the batch's
// palettes (B x K x 3) -> r = ln sum_k softmax(w)_k b_k and T = softplus(h_T), written to the
// planes ro (3 channels) and To (K + 1 channels) when given; with targets
// (planar B x 3 x H x W and B x (K + 1) x H x W), the mean-squared-error loss
// as FP64 block partials and dL/dh (bf16 NHWC, Ch channels, zero padding);
// lw = the loss weights of r, T_0 and T_1..T_K.  Written indirect values
// T_1..T_K below tk_zero are written as 0 (the loss uses the network value).
__global__ void k_head(const float* __restrict__ h, int Ch, const float* __restrict__ palette, int K, int B, int H,
                       int W, float* __restrict__ ro, Planes rop, float* __restrict__ To, Planes Top,
                       const float* __restrict__ r_t, const float* __restrict__ T_t, bf16* __restrict__ gh,
                       double* __restrict__ lossp, float3 lw, float tk_zero) {
  const long P = (long)B * H * W, HW = (long)H * W;
  const long p = (long)blockIdx.x * blockDim.x + threadIdx.x;
  float l = 0.f;
  if (p < P) {
    const Pix q = pix_of(p, H, W);
    const long o = (long)q.y * W + q.x;
    const float* hp = h + p * Ch;
    const float* pal = palette + (long)q.b * K * 3;
    float mx = -3.0e38f;
    for (int k = 0; k < K; k++) mx = fmaxf(mx, hp[k]);
    float s[16], den = 0.f;
    for (int k = 0; k < K; k++) {
      s[k] = expf(hp[k] - mx);
      den += s[k];
    }
    const float inv = 1.f / den;
    float R[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < K; k++) {
      s[k] *= inv;
      for (int c = 0; c < 3; c++) R[c] += s[k] * pal[k * 3 + c];
    }
    const float nr = 3.f * (float)P, nT = (float)(K + 1) * (float)P;
    float gR[3] = {0.f, 0.f, 0.f};
    for (int c = 0; c < 3; c++) {
      const float r = logf(R[c]);
      if (ro) ro[q.b * rop.bs + c * rop.cs + (long)q.y * rop.rs + q.x] = r;
      if (r_t) {
        const float d = r - r_t[((long)q.b * 3 + c) * HW + o];
        l += lw.x * d * d / nr;
        gR[c] = lw.x * 2.f * d / nr / R[c];
      }
    }
    for (int k = 0; k <= K; k++) {
      // T = softplus(h) = max(h, 0) + ln(1 + exp(-|h|)): non-negative layers with a
      // gradient everywhere (d softplus / dh = sigmoid(h))
      const float hk = hp[K + k], ex = expf(-fabsf(hk));
      const float t = fmaxf(hk, 0.f) + log1pf(ex);
      const float sg = hk >= 0.f ? 1.f / (1.f + ex) : ex / (1.f + ex);
      if (To) To[q.b * Top.bs + k * Top.cs + (long)q.y * Top.rs + q.x] = (k && t < tk_zero) ? 0.f : t;
      if (T_t) {
        const float d = t - T_t[((long)q.b * (K + 1) + k) * HW + o], wk = k ? lw.z : lw.y;
        l += wk * d * d / nT;
        gh[p * Ch + K + k] = __float2bfloat16(sg * wk * 2.f * d / nT);
      }
    }
    if (r_t) {
      // R_c = sum_j s_j b_jc and ds_k / dw_l = s_k (delta_kl - s_l)
      float gs[16], dot = 0.f;
      for (int k = 0; k < K; k++) {
        gs[k] = gR[0] * pal[k * 3] + gR[1] * pal[k * 3 + 1] + gR[2] * pal[k * 3 + 2];
        dot += gs[k] * s[k];
      }
      for (int k = 0; k < K; k++) gh[p * Ch + k] = __float2bfloat16(s[k] * (gs[k] - dot));
      for (int c = 2 * K + 1; c < Ch; c++) gh[p * Ch + c] = __float2bfloat16(0.f);
    }
  }
  if (!lossp) return;
  __shared__ double sh[32];
  double v = l;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); i++) t += sh[i];
    lossp[blockIdx.x] = t;
  }
}

// One Adam step on the flat FP32 master weights; c1 = 1 - b1^t, c2 = 1 - b2^t.
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long n, float lr, float b1, float b2, float eps, float c1, float c2) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi, vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// FP32 master [Co][taps][Ci] -> bf16 forward weights (same layout) and input-
// gradient weights wt[ci][taps - 1 - tap][co] (taps flipped, channels swapped).
__global__ void k_pack_weights(const float* __restrict__ w32, bf16* __restrict__ wb, bf16* __restrict__ wt, int Co,
                               int taps, int Ci) {
  const long n = (long)Co * taps * Ci;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int ci = (int)(i % Ci), tap = (int)((i / Ci) % taps), co = (int)(i / ((long)Ci * taps));
  const bf16 v = __float2bfloat16(w32[i]);
  wb[i] = v;
  wt[((long)ci * taps + (taps - 1 - tap)) * Co + co] = v;
}

}  // namespace gidnet
