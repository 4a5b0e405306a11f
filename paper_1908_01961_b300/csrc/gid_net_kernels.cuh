// Kernels of the warm-start encoder-decoder (BF16 tensor cores, FP32 accumulate).
//
// Activations are NHWC bfloat16, pixel-major (p = (b H + y) W + x) with the
// channel count a multiple of 16.  Weights are [C_out][tap][C_in] bfloat16
// (taps = 9 for 3x3, 1 for 1x1), packed from FP32 master weights.
//
// A convolution is an implicit GEMM, M = pixels, N = output channels,
// K = taps x input channels, issued as mma.sync m16n8k16 (bf16 in, fp32
// accumulate) on tiles staged in shared memory by cp.async (double buffered)
// and read with ldmatrix.  The input may be the channel concatenation of two
// tensors (the decoder's skip connections), the first of them read through a
// nearest 2x upsampling (so the upsampled tensor is never stored); the output
// may be split into two tensors (the gradient of such a concatenation).  The
// input gradient is the same kernel on the output gradient with the weights
// flipped in space and transposed in channels.  The weight gradient is a GEMM
// over pixels (M = output channels, N = taps x input channels) split across
// blocks and reduced with FP32 atomics.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gidnet {

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma16816(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void ldsm_x4(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

__device__ __forceinline__ void ldsm_x4_t(uint32_t* r, const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}

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

constexpr int CONV_BM = 128, CONV_BK = 32, CONV_LD = CONV_BK + 8;

// Block: 128 pixels x 32 WN output channels, 4 WN warps (4 along pixels, WN
// along channels), each warp 32 pixels x 32 channels (2 x 4 mma tiles).
// Grid (ceil(P / 128), (Co1 + Co2) / (32 WN)).
template <int WN>
__global__ void __launch_bounds__(128 * WN) k_conv(ConvArgs a) {
  constexpr int NT = 128 * WN, BN = 32 * WN;
  __shared__ __align__(16) bf16 sA[2][CONV_BM][CONV_LD];
  __shared__ __align__(16) bf16 sB[2][BN][CONV_LD];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int wm = warp & 3, wn = warp >> 2;
  const long P = (long)a.B * a.H * a.W;
  const long p0 = (long)blockIdx.x * CONV_BM;
  const int co0 = blockIdx.y * BN, Ci = a.C1 + a.C2, Co = a.Co1 + a.Co2;
  const int nchunk = (Ci + CONV_BK - 1) / CONV_BK, nsteps = a.taps * nchunk;

  // this thread's A rows (pixel, 16-byte chunk) for staging
  constexpr int AJ = CONV_BM * 4 / NT;
  Pix ap[AJ];
  bool aok[AJ];
#pragma unroll
  for (int j = 0; j < AJ; j++) {
    const long p = p0 + ((tid + j * NT) >> 2);
    aok[j] = p < P;
    ap[j] = pix_of(aok[j] ? p : 0, a.H, a.W);
  }

  auto stage = [&](int s, int buf) {
    const int tap = s / nchunk, ci0 = (s - tap * nchunk) * CONV_BK;
    const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
#pragma unroll
    for (int j = 0; j < AJ; j++) {
      const int i = tid + j * NT, row = i >> 2, ch = ci0 + (i & 3) * 8;
      const int yy = ap[j].y + dy, xx = ap[j].x + dx;
      const bool ok = aok[j] && ch < Ci && yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
      const bf16* src = a.in1;
      if (ok) {
        if (ch < a.C1)
          src = a.in1 + tensor_off(ap[j].b, yy, xx, a.H, a.W, a.up1, a.C1, ch);
        else
          src = a.in2 + tensor_off(ap[j].b, yy, xx, a.H, a.W, 0, a.C2, ch - a.C1);
      }
      cp16(&sA[buf][row][(i & 3) * 8], src, ok ? 16 : 0);
    }
    for (int i = tid; i < BN * 4; i += NT) {
      const int n = i >> 2, ch = ci0 + (i & 3) * 8;
      const bool ok = ch < Ci;
      const bf16* src = ok ? a.w + ((long)(co0 + n) * a.taps + tap) * Ci + ch : a.w;
      cp16(&sB[buf][n][(i & 3) * 8], src, ok ? 16 : 0);
    }
    cp_commit();
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[i][j][e] = 0.f;

  stage(0, 0);
  for (int s = 0; s < nsteps; s++) {
    const int buf = s & 1;
    if (s + 1 < nsteps) {
      stage(s + 1, buf ^ 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int k0 = 0; k0 < CONV_BK; k0 += 16) {
      uint32_t A[2][4], Bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
        ldsm_x4(A[mt], &sA[buf][wm * 32 + mt * 16 + (lane & 15)][k0 + (lane >> 4) * 8]);
#pragma unroll
      for (int np = 0; np < 2; np++) {
        uint32_t r[4];
        ldsm_x4(r, &sB[buf][wn * 32 + np * 16 + (lane & 7) + ((lane >> 4) << 3)][k0 + ((lane >> 3) & 1) * 8]);
        Bf[2 * np][0] = r[0];
        Bf[2 * np][1] = r[1];
        Bf[2 * np + 1][0] = r[2];
        Bf[2 * np + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++) mma16816(acc[mt][nt], A[mt], Bf[nt]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int mt = 0; mt < 2; mt++) {
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const long p = p0 + wm * 32 + mt * 16 + g + 8 * h;
      if (p >= P) continue;
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int co = co0 + wn * 32 + nt * 8 + 2 * t4;
        float v0 = acc[mt][nt][2 * h], v1 = acc[mt][nt][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[co];
          v1 += a.bias[co + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        if (a.out32) {
          *reinterpret_cast<float2*>(a.out32 + p * Co + co) = make_float2(v0, v1);
        } else if (co < a.Co1) {
          if (a.mask) {
            const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162*>(a.mask + p * a.Co1 + co);
            if (!(bf(m.x) > 0.f)) v0 = 0.f;
            if (!(bf(m.y) > 0.f)) v1 = 0.f;
          }
          *reinterpret_cast<uint32_t*>(a.out1 + p * a.Co1 + co) = pack2(v0, v1);
        } else {
          *reinterpret_cast<uint32_t*>(a.out2 + p * a.Co2 + (co - a.Co1)) = pack2(v0, v1);
        }
      }
    }
  }
}

struct WgradArgs {
  const bf16* g;    // NHWC, Co channels: dL/d(conv output before the activation)
  const bf16* in1;  // the conv's input, as in ConvArgs
  const bf16* in2;
  int C1, C2, up1;
  int Co;
  float* dw;  // [Co][taps][C1 + C2] fp32, accumulated
  int B, H, W, taps;
  long chunk;  // pixels per block along grid.z (multiple of 32)
};

constexpr int WG_BK = 32;

// dW[co][tap][ci] += sum_p g[p][co] in[p + offset(tap)][ci], as a GEMM with
// M = co, N = n = tap * Ci + ci, K = pixels.  Block: 32 WM output channels x
// 32 (4 / WM) columns n, 4 warps of 32 x 32; grid (Co / (32 WM), ceil(taps Ci /
// BNW), splits) with `chunk` pixels per split.
template <int WM>
__global__ void __launch_bounds__(128) k_wgrad(WgradArgs a) {
  constexpr int BMW = 32 * WM, BNW = 32 * (4 / WM), LDA = BMW + 8, LDB = BNW + 8;
  __shared__ __align__(16) bf16 sG[2][WG_BK][LDA];
  __shared__ __align__(16) bf16 sI[2][WG_BK][LDB];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, g = lane >> 2, t4 = lane & 3;
  const int wm = warp % WM, wn = warp / WM;
  const int Ci = a.C1 + a.C2, N = a.taps * Ci;
  const int co0 = blockIdx.x * BMW, n0 = blockIdx.y * BNW;
  const long P = (long)a.B * a.H * a.W;
  const long pbeg = (long)blockIdx.z * a.chunk;
  const long pend = pbeg + a.chunk < P ? pbeg + a.chunk : P;
  if (pbeg >= pend) return;
  const int nsteps = (int)((pend - pbeg + WG_BK - 1) / WG_BK);

  auto stage = [&](int s, int buf) {
    const long pc = pbeg + (long)s * WG_BK;
    for (int i = tid; i < WG_BK * (BMW / 8); i += 128) {
      const int r = i / (BMW / 8), c = (i % (BMW / 8)) * 8;
      const long p = pc + r;
      const bool ok = p < pend;
      cp16(&sG[buf][r][c], ok ? a.g + p * a.Co + co0 + c : a.g, ok ? 16 : 0);
    }
    for (int i = tid; i < WG_BK * (BNW / 8); i += 128) {
      const int r = i / (BNW / 8), c = (i % (BNW / 8)) * 8;
      const long p = pc + r;
      const int n = n0 + c;
      bool ok = p < pend && n < N;
      const bf16* src = a.in1;
      if (ok) {
        const int tap = n / Ci, ch = n - tap * Ci;
        const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
        const Pix q = pix_of(p, a.H, a.W);
        const int yy = q.y + dy, xx = q.x + dx;
        ok = yy >= 0 && yy < a.H && xx >= 0 && xx < a.W;
        if (ok)
          src = ch < a.C1 ? a.in1 + tensor_off(q.b, yy, xx, a.H, a.W, a.up1, a.C1, ch)
                          : a.in2 + tensor_off(q.b, yy, xx, a.H, a.W, 0, a.C2, ch - a.C1);
      }
      cp16(&sI[buf][r][c], src, ok ? 16 : 0);
    }
    cp_commit();
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; i++)
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
      for (int e = 0; e < 4; e++) acc[i][j][e] = 0.f;

  stage(0, 0);
  for (int s = 0; s < nsteps; s++) {
    const int buf = s & 1;
    if (s + 1 < nsteps) {
      stage(s + 1, buf ^ 1);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int k0 = 0; k0 < WG_BK; k0 += 16) {
      uint32_t A[2][4], Bf[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
        ldsm_x4_t(A[mt], &sG[buf][k0 + (lane & 7) + ((lane >> 4) << 3)][wm * 32 + mt * 16 + ((lane >> 3) & 1) * 8]);
#pragma unroll
      for (int np = 0; np < 2; np++) {
        uint32_t r[4];
        ldsm_x4_t(r, &sI[buf][k0 + (lane & 7) + ((lane >> 3) & 1) * 8][wn * 32 + np * 16 + (lane >> 4) * 8]);
        Bf[2 * np][0] = r[0];
        Bf[2 * np][1] = r[1];
        Bf[2 * np + 1][0] = r[2];
        Bf[2 * np + 1][1] = r[3];
      }
#pragma unroll
      for (int mt = 0; mt < 2; mt++)
#pragma unroll
        for (int nt = 0; nt < 4; nt++) mma16816(acc[mt][nt], A[mt], Bf[nt]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int mt = 0; mt < 2; mt++)
#pragma unroll
    for (int h = 0; h < 2; h++) {
      const int co = co0 + wm * 32 + mt * 16 + g + 8 * h;
#pragma unroll
      for (int nt = 0; nt < 4; nt++) {
        const int n = n0 + wn * 32 + nt * 8 + 2 * t4;
        if (n < N) atomicAdd(a.dw + (long)co * N + n, acc[mt][nt][2 * h]);
        if (n + 1 < N) atomicAdd(a.dw + (long)co * N + n + 1, acc[mt][nt][2 * h + 1]);
      }
    }
}

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
