// Device kernels of the illumination decomposition solver (sm_103a).
//
// Unknowns per pixel (V = K + 4): r_R, r_G, r_B (r = ln R) and T_0..T_K, stored
// as V float32 planes [V][H][pitch] (pitch a multiple of 32 floats, 128-byte
// rows).  One thread owns one pixel (or a column of pixels) in the stencil
// kernels; blocks are 32 x 8; the element-wise PCG step works on float4.
//
// The Gauss-Newton normal matrix J^T J of the IRLS-reweighted energy
// (eq:giv-energy, Sec. 5.3, Sec. 6) is never stored: every kernel that needs it
// recomputes the reweighting constants and the data-term coefficients from the
// linearisation point X and its 1-pixel halo, and the consistency pairs reach
// at most 3 pixels.  Dot products are accumulated per thread in FP32, reduced
// across the block in FP64 (warp shuffles + shared memory), and across the grid
// by the last block to finish (fixed order, so every run gives the same bits);
// the PCG scalars alpha and beta are FP64 and live in device memory, so a whole
// frame runs without a host round trip.
#pragma once

#include <cuda.h>  // CUtensorMap
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gid.h"

namespace gid {

constexpr int BX = 32, BY = 8, NT = BX * BY;
// X tile of the linearisation: BY + 6 rows, BX + 8 columns (pairs reach 3, rows
// of 40 floats = 160 bytes keep every TMA row 16-byte aligned)
constexpr int LIN_R = BY + 6, LIN_C = BX + 8;

struct Weights {
  float ld, lcl, lrs, p, lrc, lm, lis, lsm, lnn, lIR, lCR, eps, sharp, tau;
  int nonneg_strict, irls_half, rcluster_follows_b;
};

// Base colours: current (refined) b_1..b_K, the initial estimate, FP64 master.
struct DevColors {
  float b[GID_MAX_K * 3];
  float binit[GID_MAX_K * 3];
  double bd[GID_MAX_K * 3];
};

enum : int { ST_BAD_LABEL = 1, ST_SINGULAR = 2, ST_TIMEOUT = 4 };

struct DevScalars {
  double rho, pq, alpha, beta;
  double rho2[2];  // rho of PCG step m in slot m % 2 (see k_apply)
  double energy[8];
  double A[3 * GID_MAX_K * GID_MAX_K];
  double g[3 * GID_MAX_K];
  unsigned int cnt[8];
  int status;
  // host-side fault injection (gid_debug_inject; zero = off): participants of
  // the persistent kernel's grid barrier that never arrive, and the barrier's
  // poll limit (0 = GRID_SPINS)
  unsigned int phantom;
  long long spin_limit;
  // rho_m = <r_m, z_m> of the latest Gauss-Newton step, m = 0 .. min(M, PCG_HIST) - 1
  // (slot 0 by the PCG start; the others copied from rho2 when recording is on)
  double rho_hist[64];
};
constexpr int PCG_HIST = 64;
// arrival counters: linearisation, base-colour step per colour channel (3),
// energy, persistent-kernel grid barrier (count, generation)
enum { CNT_LIN, CNT_DENSE, CNT_ENERGY = CNT_DENSE + 3, CNT_GRID, CNT_GEN };

struct Params {
  int H, W, pitch;
  long plane;
  Weights w;
  const float* I;
  const uint8_t* lab;
  const float* wsr;
  const float* ws;     // n_s planes: spatial pair weights omega_j(x), 0 if x + o_j is outside
  const float* wt;     // n_t planes: temporal pair weights
  const float* wtsum;  // sum_j of the temporal weights
  const float* rprev;  // 3 planes
  int ns, nt, temporal;
  int off_s[2 * GID_MAX_PAIRS];
  int off_t[2 * GID_MAX_PAIRS];
  float* X;
  float* d;
  float* z;
  float* q;
  float* Minv;
  float* coef;  // operator coefficient planes written by k_linearize (CoefLayout)
  float* blk;   // block-Jacobi blocks in Schur form, block_planes(K) planes (k_block_factor)
  DevColors* col;
  DevScalars* sc;
  double* partial;
  double* pcg_part;  // [2 kinds: operator <p,q>, vector <r,z>][2 parities][nbmax] block partials
  int nbmax;
  // resident PCG kernel: border exchange planes (2 x V planes, pitched) and the
  // grid all-reduce slots [RES_ROWS][RES_NV][RES_MAXB] followed by the arrival
  // counters (RES_ROWS, each on its own 128-byte line)
  float* zx;
  double* xval;
};
// most blocks of one resident PCG launch (one per SM)
constexpr int RES_MAXB = 1024;
constexpr int RES_ROWS = 4, RES_NV = 3;

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ int tid_flat() { return threadIdx.y * blockDim.x + threadIdx.x; }

// FP64 arithmetic runs at a small fraction of the FP32 rate on this part (a
// warp-wide FP64 add holds the FP64 pipe for many cycles), so every block
// reduction below does its FP64 additions in warp 0 only: a 5-level shuffle
// tree over at most 32 values, in a fixed order.

// FP64 shuffle tree over warp 0 (the caller is warp 0); the sum in lane 0.
__device__ __forceinline__ double warp_tree(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block sum of per-thread FP32 partials: an FP32 shuffle tree inside each warp
// (32 terms, pairwise), then the warp sums added in FP64 by warp 0's tree.
// Valid in thread 0.  All threads call.
__device__ __forceinline__ double block_sum_f(float v) {
  __shared__ float sh[32];
  const int t = tid_flat(), lane = t & 31, wid = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) s = warp_tree(lane < nw ? (double)sh[lane] : 0.0);
  __syncthreads();
  return s;
}

// True in every thread of the last block to arrive.  Thread 0 must have
// written this block's partials before the call.  Resets the counter.
__device__ __forceinline__ bool last_block(unsigned int* cnt, unsigned int n = 0u) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (tid_flat() == 0) {
    if (n == 0u) n = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int t = atomicAdd(cnt, 1u);
    is_last = (t == n - 1);
    if (is_last) *cnt = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// The PCG scalars are formed by the kernel that consumes them: every block sums
// the previous kernel's block partials in the same fixed order (so all blocks
// agree bit for bit), and no kernel of the PCG loop has a serial last-block
// tail.  part_share: lane l of warp 0 adds part[l], part[l + 32], ... (its
// loads may be issued early; 0 in the other warps); block_total: warp 0's tree
// of those shares, returned to every thread of the block.
__device__ __forceinline__ double part_share(const double* part, int n) {
  double s = 0.0;
  const int t = tid_flat();
  if (t < 32)
    for (int i = t; i < n; i += 32) s += __ldcg(part + i);
  return s;
}

__device__ __forceinline__ double block_total(double v) {
  __shared__ double tot;
  const int t = tid_flat();
  if (t < 32) {
    v = warp_tree(v);
    if (t == 0) tot = v;
  }
  __syncthreads();
  const double r = tot;
  __syncthreads();
  return r;
}

// Sum of n partials (stride `stride`, starting at `base`) in a fixed order,
// valid in thread 0: lane l of warp 0 adds partials l, l + 32, ... into four
// interleaved accumulators (loads in flight together), combined in order.
__device__ __forceinline__ double grid_total(const double* partial, int n, int stride, int base) {
  double s = 0.0;
  const int t = tid_flat();
  if (t < 32) {
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    int i = t;
    for (; i + 96 < n; i += 128) {
#pragma unroll
      for (int u = 0; u < 4; u++) a[u] += __ldcg(partial + (long)(i + 32 * u) * stride + base);
    }
    for (; i < n; i += 32) a[0] += __ldcg(partial + (long)i * stride + base);
    s = warp_tree((a[0] + a[1]) + (a[2] + a[3]));
  }
  __syncthreads();
  return s;
}

__device__ __forceinline__ double* pcg_partials(const Params& P, int kind, int it) {
  return P.pcg_part + ((long)kind * 2 + (it & 1)) * P.nbmax;
}
// kinds: <p, q> (operator step), <r, z> (vector step); the fused PCG step
// (k_pcg_step) uses <p, q>, <z, q> in the second kind's slots and <q, M^-1 q>
enum { PART_PQ = 0, PART_RZ = 1, PART_ZQ = 1, PART_QMQ = 2, PART_KINDS = 3 };

// ---------------------------------------------------------------- IRLS weights (Sec. 5.3)

__device__ __forceinline__ float irls_l1(const Weights& w, float lambda, float g) {
  float v = lambda / (fabsf(g) + w.eps);
  return w.irls_half ? 0.5f * v : v;
}

__device__ __forceinline__ float irls_lp(const Weights& w, float lambda, float gnorm) {
  float v = (w.p == 1.0f) ? lambda / (gnorm + w.eps) : lambda * powf(gnorm + w.eps, w.p - 2.0f);
  return w.irls_half ? 0.5f * v : v;
}

// lambda_nonneg * w_k of Sec. 5.3.1 (0 for T > 0, or T >= 0 unless strict).
__device__ __forceinline__ float nonneg_weight(const Weights& w, float T) {
  bool free_ = w.nonneg_strict ? (T > 0.0f) : (T >= 0.0f);
  float v = free_ ? 0.0f : w.lnn / (fabsf(T) + w.eps);
  return w.irls_half ? 0.5f * v : v;
}

// ---------------------------------------------------------------- per-block colour tables

template <int K>
struct ColorTable {
  float b[K + 1][3];   // b_0 = white, b_1..b_K current
  float dm[K + 1][3];  // b_kc - mean_c' b_kc' (monochrome prior Jacobian)
  float bi[K + 1][3];  // initial estimate (b_0 white)
};

template <int K>
__device__ __forceinline__ void load_colors(ColorTable<K>& t, const DevColors* col) {
  const int i = tid_flat();
  if (i < K + 1) {
    float m = 0.f;
    for (int c = 0; c < 3; c++) {
      float v = i == 0 ? 1.0f : col->b[(i - 1) * 3 + c];
      t.b[i][c] = v;
      t.bi[i][c] = i == 0 ? 1.0f : col->binit[(i - 1) * 3 + c];
      m += v;
    }
    m *= (1.0f / 3.0f);
    for (int c = 0; c < 3; c++) t.dm[i][c] = t.b[i][c] - m;
  }
  __syncthreads();
}

// ---------------------------------------------------------------- operator coefficients

// Per-pixel coefficients of J^T J at the linearisation point, one plane each,
// written once per Gauss-Newton step by k_linearize and read by every PCG
// operator step of that step:
//   A  (3)     lambda_data R_c^2                  data term
//   S  (3)     S_c = sum_k b_kc T_k               data term
//   WR, WD     r-sparsity weight of the edge to the right / below (0 if absent)
//   ER, ED     smoothness weight of each layer's edge to the right / below (0 if absent)
//   WT (K+1)   non-negativity + decomposition-sparsity diagonal of each layer
//   DR         lambda_clustering + temporal consistency diagonal of r
//   WM         lambda_monochrome w_SR
//   CW + j     lambda_r-consistency omega_j(x): pair (x, x + o_j), 0 if x + o_j is outside
//   CW + ns + j  lambda_r-consistency omega_j(x - o_j): pair (x - o_j, x), 0 if x - o_j is outside
template <int K>
struct CoefLayout {
  static constexpr int A = 0, S = 3, WR = 6, WD = 7, ER = 8, ED = 8 + (K + 1), WT = 8 + 2 * (K + 1),
                       DR = 8 + 3 * (K + 1), WM = 9 + 3 * (K + 1), CW = 10 + 3 * (K + 1);
};
constexpr int coef_planes(int K, int ns) { return 10 + 3 * (K + 1) + 2 * ns; }

// ---- TMA: one elected thread copies a 3-D box of planes into shared memory,
// completion counted in bytes on an mbarrier.
constexpr long TMA_SPINS = 1L << 22;  // bounded wait (then ST_TIMEOUT)

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Box of the tensor map at (x, y, z) (x in elements, 16-byte aligned; may be
// negative or past the end: those elements read as zero).
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];\n" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// ---------------------------------------------------------------- stencil helpers

struct Pix {
  int x, y;
  bool hR, hD, hL, hU;  // neighbour exists: right, down, left, up
};

__device__ __forceinline__ Pix make_pix(const Params& P, int x, int y) {
  return Pix{x, y, x + 1 < P.W, y + 1 < P.H, x > 0, y > 0};
}

__device__ __forceinline__ long off2(const Params& P, int y, int x) { return (long)y * P.pitch + x; }

__device__ __forceinline__ bool inside(const Params& P, int y, int x) {
  return (unsigned)y < (unsigned)P.H && (unsigned)x < (unsigned)P.W;
}

// IRLS weight of the reflectance gradient at pixel (y, x) (forward differences
// over the three log channels, missing components zero).
__device__ __forceinline__ float rsparse_weight(const Params& P, const float* __restrict__ X, int y, int x) {
  const long o = off2(P, y, x);
  float g2 = 0.f;
  if (x + 1 < P.W)
    for (int c = 0; c < 3; c++) {
      float dd = X[c * P.plane + o + 1] - X[c * P.plane + o];
      g2 += dd * dd;
    }
  if (y + 1 < P.H)
    for (int c = 0; c < 3; c++) {
      float dd = X[c * P.plane + o + P.pitch] - X[c * P.plane + o];
      g2 += dd * dd;
    }
  return irls_lp(P.w, P.w.lrs, sqrtf(g2));
}

// Edge weights of the four edges touching pixel px for the r-sparsity term.
struct Edges {
  float R, D, L, U;
};

__device__ __forceinline__ Edges rsparse_edges(const Params& P, const float* __restrict__ X, const Pix& px) {
  float wc = rsparse_weight(P, X, px.y, px.x);
  Edges e;
  e.R = px.hR ? wc : 0.f;
  e.D = px.hD ? wc : 0.f;
  e.L = px.hL ? rsparse_weight(P, X, px.y, px.x - 1) : 0.f;
  e.U = px.hU ? rsparse_weight(P, X, px.y - 1, px.x) : 0.f;
  return e;
}

// Smoothness edge weights of layer plane v (Sec. 5.2, anisotropic l1).
__device__ __forceinline__ Edges smooth_edges(const Params& P, const float* __restrict__ X, int v, const Pix& px,
                                              float tc) {
  const float* t = X + v * P.plane + off2(P, px.y, px.x);
  Edges e;
  e.R = px.hR ? irls_l1(P.w, P.w.lsm, t[1] - tc) : 0.f;
  e.D = px.hD ? irls_l1(P.w, P.w.lsm, t[P.pitch] - tc) : 0.f;
  e.L = px.hL ? irls_l1(P.w, P.w.lsm, tc - t[-1]) : 0.f;
  e.U = px.hU ? irls_l1(P.w, P.w.lsm, tc - t[-P.pitch]) : 0.f;
  return e;
}

// sum over existing edges of w_e (f(x) - f(neighbour)).  f is a functor f(dy, dx).
template <class F>
__device__ __forceinline__ float edge_laplace(const Edges& e, const Pix& px, float fc, F f) {
  float s = 0.f;
  if (px.hR) s += e.R * (fc - f(0, 1));
  if (px.hD) s += e.D * (fc - f(1, 0));
  if (px.hL) s += e.L * (fc - f(0, -1));
  if (px.hU) s += e.U * (fc - f(-1, 0));
  return s;
}

// ---------------------------------------------------------------- kernels

// Frame ingest: planar contiguous rgb/labels -> pitched I, labels, chromaticity C.
__global__ void k_ingest(Params P, const float* __restrict__ rgb, const uint8_t* __restrict__ labels, int K,
                         float* __restrict__ C, uint8_t* __restrict__ lab_out, float* __restrict__ I_out) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  const long src = (long)y * P.W + x, HW = (long)P.H * P.W, o = off2(P, y, x);
  float v[3];
  for (int c = 0; c < 3; c++) v[c] = rgb[c * HW + src];
  const float s = v[0] + v[1] + v[2] + 1e-6f;
  for (int c = 0; c < 3; c++) {
    I_out[c * P.plane + o] = v[c];
    C[c * P.plane + o] = v[c] / s;
  }
  uint8_t l = labels[src];
  if (l >= K) {
    atomicOr(&P.sc->status, ST_BAD_LABEL);
    l = 0;
  }
  lab_out[o] = l;
}

// Soft-Retinex weight (Sec. 5.2) and consistency pair weights.
__global__ void k_prior_weights(Params P, const float* __restrict__ C, const float* __restrict__ Cprev,
                                float* __restrict__ wsr, float* __restrict__ ws, float* __restrict__ wt,
                                float* __restrict__ wtsum) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  const long o = off2(P, y, x);
  float cc[3];
  for (int c = 0; c < 3; c++) cc[c] = C[c * P.plane + o];
  auto dist2 = [&](const float* Cb, int yy, int xx) {
    const long n = off2(P, yy, xx);
    float s = 0.f;
    for (int c = 0; c < 3; c++) {
      float dd = Cb[c * P.plane + n] - cc[c];
      s += dd * dd;
    }
    return s;
  };
  float dmax = 0.f;
  const int N4[4][2] = {{0, 1}, {0, -1}, {1, 0}, {-1, 0}};
  for (int n = 0; n < 4; n++) {
    int yy = y + N4[n][0], xx = x + N4[n][1];
    if (inside(P, yy, xx)) dmax = fmaxf(dmax, sqrtf(dist2(C, yy, xx)));
  }
  wsr[o] = 1.0f - expf(-P.w.sharp * dmax);
  const float it2 = 1.0f / (P.w.tau * P.w.tau);
  for (int j = 0; j < P.ns; j++) {
    int yy = y + P.off_s[2 * j], xx = x + P.off_s[2 * j + 1];
    ws[j * P.plane + o] = inside(P, yy, xx) ? expf(-dist2(C, yy, xx) * it2) : 0.f;
  }
  if (P.temporal) {
    float s = 0.f;
    for (int j = 0; j < P.nt; j++) {
      int yy = y + P.off_t[2 * j], xx = x + P.off_t[2 * j + 1];
      float v = inside(P, yy, xx) ? expf(-dist2(Cprev, yy, xx) * it2) : 0.f;
      wt[j * P.plane + o] = v;
      s += v;
    }
    wtsum[o] = s;
  }
}

// Refined base colours back to the initial estimate.
__global__ void k_reset_colors(DevColors* col, int n) {
  const int i = threadIdx.x;
  if (i < n) {
    col->b[i] = col->binit[i];
    col->bd[i] = (double)col->binit[i];
  }
}

// Cold start: r = ln R_cluster, T_0 = mean_c I / mean_c R_cluster, T_k = 0.
template <int K>
__global__ void k_init_cold(Params P) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (y >= P.H || x >= P.pitch) return;
  const long o = off2(P, y, x);
  if (x >= P.W) {  // padding columns are zero (a failed earlier solve may have left NaN there)
#pragma unroll
    for (int v = 0; v < K + 4; v++) P.X[v * P.plane + o] = 0.f;
    return;
  }
  const int l = P.lab[o];
  const float* bsrc = P.w.rcluster_follows_b ? P.col->b : P.col->binit;
  float mi = 0.f, mr = 0.f;
  for (int c = 0; c < 3; c++) {
    float bc = bsrc[l * 3 + c];
    P.X[c * P.plane + o] = logf(bc);
    mi += P.I[c * P.plane + o];
    mr += bc;
  }
  P.X[3 * P.plane + o] = mi / mr;
  for (int k = 1; k <= K; k++) P.X[(3 + k) * P.plane + o] = 0.f;
}

// T_0 minimising the data term (eq:data-term) per pixel with r, T_1..T_K and
// the current b fixed: sum_c R_c (I_c - R_c A_c) / sum_c R_c^2 with
// A_c = sum_k b_kc T_k, taken at 0 when negative.
template <int K>
__global__ void k_fit_direct(Params P) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  const long o = off2(P, y, x);
  float T[K + 1];
#pragma unroll
  for (int k = 1; k <= K; k++) T[k] = P.X[(3 + k) * P.plane + o];
  float num = 0.f, den = 0.f;
  for (int c = 0; c < 3; c++) {
    const float R = expf(P.X[c * P.plane + o]);
    float A = 0.f;
#pragma unroll
    for (int k = 1; k <= K; k++) A += P.col->b[(k - 1) * 3 + c] * T[k];
    num += R * (P.I[c * P.plane + o] - R * A);
    den += R * R;
  }
  P.X[3 * P.plane + o] = fmaxf(num / den, 0.f);
}

// Shared per-pixel state at the linearisation point.
template <int K>
struct PixState {
  float rr[3], T[K + 1], R[3], S[3];
};

template <int K>
__device__ __forceinline__ void load_state(const Params& P, const ColorTable<K>& ct, long o, PixState<K>& s) {
  for (int c = 0; c < 3; c++) s.rr[c] = P.X[c * P.plane + o];
#pragma unroll
  for (int k = 0; k <= K; k++) s.T[k] = P.X[(3 + k) * P.plane + o];
  for (int c = 0; c < 3; c++) {
    s.R[c] = expf(s.rr[c]);
    float v = 0.f;
#pragma unroll
    for (int k = 0; k <= K; k++) v += ct.b[k][c] * s.T[k];
    s.S[c] = v;
  }
}

// Linearisation (fused): g = -J^T F, diag(J^T J); PCG start z = M^-1 g (the
// residual r = g itself is not stored);
// the operator coefficients of the step (CoefLayout) in every mode.
// mode 0: PCG init (writes z, Minv, zero delta, rho); mode 1: stage output
// (writes g to gout and diag to dout); mode 2: coefficients only; mode 3:
// block-Jacobi start (writes g to z, diag to Minv, zero delta; k_block_factor
// completes the PCG init).
template <int K>
__global__ void __launch_bounds__(NT, K <= 6 ? 4 : 1) k_linearize(Params P, int mode, float* __restrict__ gout,
                                                  float* __restrict__ dout,
                                                  const __grid_constant__ CUtensorMap mapX) {
  constexpr int V = K + 4;
  __shared__ ColorTable<K> ct;
  // the block's tile of X with the consistency pairs' reach: rows y0 - 3 ..
  // y0 + BY + 2, columns x0 - 4 .. x0 + BX + 3 (one TMA box, zero outside)
  __shared__ alignas(128) float sX[V][LIN_R][LIN_C];
  __shared__ __align__(8) uint64_t bar;
  load_colors<K>(ct, P.col);
  const int x0 = blockIdx.x * BX, y0 = blockIdx.y * BY;
  if (tid_flat() == 0) mbar_init(&bar, 1);
  __syncthreads();
  if (tid_flat() == 0) {
    mbar_expect_tx(&bar, (unsigned)sizeof(sX));
    tma_load_3d(&sX[0][0][0], &mapX, x0 - 4, y0 - 3, 0, &bar);
  }
  bool staged = false;
  for (long i = 0; i < TMA_SPINS && !staged; i++) staged = mbar_try_wait(&bar, 0);
  if (!__syncthreads_and(staged)) {
    // the copy did not complete in time: record it and give the copy still in
    // flight into this block's shared memory a second bounded wait; the block
    // then writes no state (its partial of rho is zero, so the grid reduction
    // below still counts every block)
    if (tid_flat() == 0) atomicOr(&P.sc->status, ST_TIMEOUT);
    for (long i = 0; i < TMA_SPINS && !staged; i++) staged = mbar_try_wait(&bar, 0);
    staged = false;
  }
  // X reads go to the tile: the same indexing helpers with the tile's strides
  // and a base that maps absolute (y, x) into it
  Params Q = P;
  Q.pitch = LIN_C;
  Q.plane = (long)LIN_R * LIN_C;
  Q.X = &sX[0][0][0] - ((long)(y0 - 3) * LIN_C + (x0 - 4));
  const Weights& w = P.w;
  const int x = x0 + threadIdx.x, y = y0 + threadIdx.y;
  float rz = 0.f;
  // the resident PCG launch that follows starts with cleared arrival counters
  if (P.xval && blockIdx.x == 0 && blockIdx.y == 0 && tid_flat() < 32 * RES_ROWS)
    reinterpret_cast<unsigned int*>(P.xval + (long)RES_ROWS * RES_NV * RES_MAXB)[tid_flat()] = 0u;
  if ((mode == 0 || mode == 3) && x >= P.W && x < P.pitch && y < P.H) {
    // the PCG vectors' padding columns restart at zero every Gauss-Newton step
    const long o = off2(P, y, x);
#pragma unroll
    for (int v = 0; v < V; v++) P.z[v * P.plane + o] = P.d[v * P.plane + o] = P.Minv[v * P.plane + o] = 0.f;
  }
  if (staged && x < P.W && y < P.H) {
    const Pix px = make_pix(P, x, y);
    const long o = off2(P, y, x), oq = off2(Q, y, x);
    PixState<K> s;
    load_state<K>(Q, ct, oq, s);
    float g[V], dg[V];
#pragma unroll
    for (int v = 0; v < V; v++) g[v] = dg[v] = 0.f;
    // Linear terms: g -= A_lin X and diag += diag(A_lin), with the same stencil
    // as normal_apply; the data term is handled separately below.
    const float* X = Q.X;
    auto xf = [&](int v, int dy, int dx) { return X[v * Q.plane + oq + (long)dy * Q.pitch + dx]; };
    // E_data: residual e_c = I_c - R_c S_c.
    for (int c = 0; c < 3; c++) {
      const float e = P.I[c * P.plane + o] - s.R[c] * s.S[c];
      g[c] += w.ld * s.R[c] * s.S[c] * e;
      dg[c] += w.ld * s.R[c] * s.R[c] * s.S[c] * s.S[c];
#pragma unroll
      for (int k = 0; k <= K; k++) {
        g[3 + k] += w.ld * s.R[c] * ct.b[k][c] * e;
        dg[3 + k] += w.ld * s.R[c] * s.R[c] * ct.b[k][c] * ct.b[k][c];
      }
    }
    // E_clustering.
    const int l = P.lab[o];
    const float* bcl = w.rcluster_follows_b ? P.col->b : P.col->binit;
    for (int c = 0; c < 3; c++) {
      g[c] -= w.lcl * (s.rr[c] - logf(bcl[l * 3 + c]));
      dg[c] += w.lcl;
    }
    // E_r-sparsity.
    const Edges er = rsparse_edges(Q, X, px);
    for (int c = 0; c < 3; c++) {
      g[c] -= edge_laplace(er, px, s.rr[c], [&](int dy, int dx) { return xf(c, dy, dx); });
      dg[c] += er.R + er.D + er.L + er.U;
    }
    // E_r-consistency, spatial.
    for (int j = 0; j < P.ns; j++) {
      const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
      float of = 0.f, ob = 0.f;
      if (inside(P, y + dy, x + dx)) {
        of = w.lrc * P.ws[j * P.plane + o];
        for (int c = 0; c < 3; c++) {
          g[c] -= of * (s.rr[c] - xf(c, dy, dx));
          dg[c] += of;
        }
      }
      if (inside(P, y - dy, x - dx)) {
        ob = w.lrc * P.ws[j * P.plane + o - (long)dy * P.pitch - dx];
        for (int c = 0; c < 3; c++) {
          g[c] -= ob * (s.rr[c] - xf(c, -dy, -dx));
          dg[c] += ob;
        }
      }
      P.coef[(CoefLayout<K>::CW + j) * P.plane + o] = of;
      P.coef[(CoefLayout<K>::CW + P.ns + j) * P.plane + o] = ob;
    }
    // E_r-consistency, temporal: residual r(x) - r_prev(x + o_j).
    if (P.temporal) {
      for (int j = 0; j < P.nt; j++) {
        const int dy = P.off_t[2 * j], dx = P.off_t[2 * j + 1];
        if (!inside(P, y + dy, x + dx)) continue;
        const float wj = w.lrc * P.wt[j * P.plane + o];
        const long n = o + (long)dy * P.pitch + dx;
        for (int c = 0; c < 3; c++) {
          g[c] -= wj * (s.rr[c] - P.rprev[c * P.plane + n]);
          dg[c] += wj;
        }
      }
    }
    // E_monochrome.
    const float wm = w.lm * P.wsr[o];
    for (int c = 0; c < 3; c++) {
      float m = 0.f;
#pragma unroll
      for (int k = 0; k <= K; k++) m += ct.dm[k][c] * s.T[k];
#pragma unroll
      for (int k = 0; k <= K; k++) {
        g[3 + k] -= wm * ct.dm[k][c] * m;
        dg[3 + k] += wm * ct.dm[k][c] * ct.dm[k][c];
      }
    }
    // E_i-sparsity and E_non-neg.
    using CL = CoefLayout<K>;
    float* cf = P.coef + o;
#pragma unroll
    for (int k = 0; k <= K; k++) {
      float wd = nonneg_weight(w, s.T[k]);
      if (k > 0) wd += irls_l1(w, w.lis, s.T[k]);
      g[3 + k] -= wd * s.T[k];
      dg[3 + k] += wd;
      cf[(CL::WT + k) * P.plane] = wd;
    }
    // E_smoothness.
#pragma unroll
    for (int k = 0; k <= K; k++) {
      const Edges es = smooth_edges(Q, X, 3 + k, px, s.T[k]);
      g[3 + k] -= edge_laplace(es, px, s.T[k], [&](int dy, int dx) { return xf(3 + k, dy, dx); });
      dg[3 + k] += es.R + es.D + es.L + es.U;
      cf[(CL::ER + k) * P.plane] = es.R;
      cf[(CL::ED + k) * P.plane] = es.D;
    }
#pragma unroll
    for (int c = 0; c < 3; c++) {
      cf[(CL::A + c) * P.plane] = w.ld * s.R[c] * s.R[c];
      cf[(CL::S + c) * P.plane] = s.S[c];
    }
    cf[CL::WR * P.plane] = er.R;
    cf[CL::WD * P.plane] = er.D;
    cf[CL::DR * P.plane] = w.lcl + (P.temporal ? w.lrc * P.wtsum[o] : 0.f);
    cf[CL::WM * P.plane] = wm;
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        const long ov = v * P.plane + o;
        const float mi = 1.0f / dg[v];
        const float zz = mi * g[v];
        P.Minv[ov] = mi;
        P.z[ov] = zz;
        P.d[ov] = 0.f;
        rz += g[v] * zz;
      }
    } else if (mode == 3) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        const long ov = v * P.plane + o;
        P.Minv[ov] = dg[v];
        P.z[ov] = g[v];
        P.d[ov] = 0.f;
      }
    } else if (mode == 1) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        const long ov = v * P.plane + o;
        gout[ov] = g[v];
        dout[ov] = dg[v];
      }
    }
  }
  if (mode != 0) return;
  const double bs = block_sum_f(rz);
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid_flat() == 0) P.partial[b] = bs;
  if (last_block(&P.sc->cnt[CNT_LIN])) {
    const double t = grid_total(P.partial, nb, 1, 0);
    if (tid_flat() == 0) {
      P.sc->rho = t;
      P.sc->rho2[1] = t;  // rho of PCG step 1
      P.sc->rho_hist[0] = t;
      P.sc->beta = 0.0;
      P.sc->cnt[CNT_GRID] = 0u;  // arrival counter of the persistent PCG kernel's grid barrier
    }
  }
}

// ---------------------------------------------------------------- PCG operator step

// ---- four pixels as two packed FP32 pairs (one packed instruction per pair)

struct F4 {
  float2 a, b;  // pixels 0,1 and 2,3
};
__device__ __forceinline__ F4 f4(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ F4 f4s(float s) { return {make_float2(s, s), make_float2(s, s)}; }
__device__ __forceinline__ F4 f4v(float x, float y, float z, float w) { return {make_float2(x, y), make_float2(z, w)}; }
__device__ __forceinline__ float4 to4(F4 v) { return make_float4(v.a.x, v.a.y, v.b.x, v.b.y); }
__device__ __forceinline__ F4 fma4(F4 x, F4 y, F4 z) { return {__ffma2_rn(x.a, y.a, z.a), __ffma2_rn(x.b, y.b, z.b)}; }
__device__ __forceinline__ F4 mul4(F4 x, F4 y) { return {__fmul2_rn(x.a, y.a), __fmul2_rn(x.b, y.b)}; }
__device__ __forceinline__ F4 add4(F4 x, F4 y) { return {__fadd2_rn(x.a, y.a), __fadd2_rn(x.b, y.b)}; }
// x - y, exactly rounded (one fused multiply-add by -1)
__device__ __forceinline__ F4 sub4(F4 x, F4 y) {
  const float2 m = make_float2(-1.f, -1.f);
  return {__ffma2_rn(y.a, m, x.a), __ffma2_rn(y.b, m, x.b)};
}
__device__ __forceinline__ float dot4(F4 x, F4 y) {
  const float2 t = __ffma2_rn(x.b, y.b, __fmul2_rn(x.a, y.a));
  return t.x + t.y;
}
__device__ __forceinline__ F4 ldg4(const float* p) { return f4(*reinterpret_cast<const float4*>(p)); }
// load through the read-only path: for data no thread of the kernel writes (the
// operator coefficients, M^-1), which frees the compiler to issue it ahead of
// the kernel's stores
__device__ __forceinline__ F4 ldc4(const float* p) { return f4(__ldg(reinterpret_cast<const float4*>(p))); }
__device__ __forceinline__ F4 lds4(const float* p) { return f4(*reinterpret_cast<const float4*>(p)); }

// Tile of the operator kernel: 128 x 8 pixels per 32 x 8 block, four
// consecutive pixels in x per thread.  p = z + beta p_old is formed once per
// position into shared memory in aligned float4 chunks: rows y0-3 .. y0+10 of
// the reflectance channels (the consistency pairs reach 3 pixels) and rows
// y0-1 .. y0+8 of the layers, columns x0-4 .. x0+131 (halo padded to a float4).
constexpr int QW = 4, VTW = BX * QW, VHX = 4, VRW = VHX + VTW + 4, AHR = 3;

// Both arrays are TMA destinations (128-byte aligned boxes: [3][TH + 6][136]
// and [K + 1][TH + 2][136] floats).
template <int K, int TH>
struct ApplyTile {
  alignas(128) float pr[3][TH + 2 * AHR][VRW];
  alignas(128) float pt[K + 1][TH + 2][VRW];
};

// Apply tile shapes: TH rows of 128 pixels, a 32 x TH block, at most MAXREG
// registers per thread (MINB blocks of it fit in one SM's register file).
template <int TH>
struct ApplyShape;
template <>
struct ApplyShape<8> {
  static constexpr int MINB = 2, MAXREG = 128;
};
template <>
struct ApplyShape<4> {
  static constexpr int MINB = 4, MAXREG = 128;
};
template <>
struct ApplyShape<2> {
  static constexpr int MINB = 8, MAXREG = 128;
};
// 17 rows, one 544-thread block per SM: a 640 x 480 frame is 145 such tiles,
// one wave on 148 SMs.  17 warps put 5 warps on one SM sub-partition (16 K
// registers), hence at most 96 registers per thread.
// 16 rows, one 512-thread block per SM at up to 128 registers (16 warps: 4 per
// sub-partition): for frames large enough that the 17-row tile's single wave
// does not matter (1920 x 1080, the batch's work list), where it also avoids
// the 96-register spills of K >= 7.
template <>
struct ApplyShape<16> {
  static constexpr int MINB = 1, MAXREG = 128;
};
template <>
struct ApplyShape<17> {
  static constexpr int MINB = 1, MAXREG = 96;
};

// q = A s at one thread's four pixels (x .. x + 3 of row y, x < W, y < H), A =
// J^T J at the Gauss-Newton step's linearisation point given by the
// coefficient planes (CoefLayout), s read from a staged tile: reflectance
// channel c at sr[c * SRC + dy * SRR + dx] and layer k at st[k * STC + dy * STR +
// dx] for the offset (dy, dx) from the first pixel (sr and st point at that
// pixel; the tile holds s with a halo of 3 rows and 4 columns for the
// reflectance channels, 1 row and 4 columns for the layers, zero outside the
// frame).  finish(v, s_v, (A s)_v) is called once per plane v (reflectance
// channels first) with the four pixels' values; lanes past the frame's right
// edge of A s are zero.  The layer loop is not unrolled: unrolled, the 2-, 4- and
// 8-row tiles spilled at 128 registers (416 bytes at K = 8) and ran 4-8 %
// slower on frames of many tiles.
// SHFL: the left neighbour's right-edge weights come from lane - 1 of the warp
// where left_lane says that lane holds the chunk to the left (every lane of the
// warp must then make the call); elsewhere they are loaded.
template <int K, bool SHFL = false, class FIN>
__device__ __forceinline__ void op_apply4(const Params& P, const ColorTable<K>& ct, int x, int y,
                                          const float* sr, int SRC, int SRR, const float* st, int STC, int STR,
                                          FIN finish, bool left_lane = false) {
  using CL = CoefLayout<K>;
  const long o = off2(P, y, x);
  const float* __restrict__ cf = P.coef + o;
  const long PL = P.plane;
  const bool hL = x > 0, hU = y > 0;
  const F4 valid = f4v(1.f, x + 1 < P.W ? 1.f : 0.f, x + 2 < P.W ? 1.f : 0.f, x + 3 < P.W ? 1.f : 0.f);
  // data block: P_c = sum_k b_kc p_Tk
  F4 u[3];
#pragma unroll
  for (int c = 0; c < 3; c++) u[c] = f4s(0.f);
#pragma unroll
  for (int k = 0; k <= K; k++) {
    const F4 pk = lds4(st + k * STC);
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma4(f4s(ct.b[k][c]), pk, u[c]);
  }
  // reflectance channels, one at a time: data, clustering/temporal diagonal,
  // r-sparsity, consistency pairs (x, x + o_j) and (x - o_j, x); the shared
  // per-pixel weights are re-read through L1 rather than held in registers
  float eLm;
  if constexpr (SHFL) {
    const float sh = __shfl_up_sync(0xffffffffu, cf[CL::WR * PL + 3], 1);
    eLm = left_lane ? sh : (hL ? cf[CL::WR * PL - 1] : 0.f);
  } else {
    eLm = hL ? cf[CL::WR * PL - 1] : 0.f;
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {
    const F4 Sc = ldg4(cf + (CL::S + c) * PL), Ac = ldg4(cf + (CL::A + c) * PL);
    const float* row = sr + c * SRC;
    const F4 pc = lds4(row);
    u[c] = mul4(Ac, fma4(Sc, pc, u[c]));  // u_c = A_c (S_c p_rc + P_c)
    F4 q = fma4(Sc, u[c], mul4(ldg4(cf + CL::DR * PL), pc));
    {
      const F4 eR = ldg4(cf + CL::WR * PL), eD = ldg4(cf + CL::WD * PL);
      const F4 eL = f4v(eLm, eR.a.x, eR.a.y, eR.b.x);
      const F4 right = f4v(pc.a.y, pc.b.x, pc.b.y, row[4]);
      const F4 left = f4v(row[-1], pc.a.x, pc.a.y, pc.b.x);
      q = fma4(eR, sub4(pc, right), q);
      q = fma4(eL, sub4(pc, left), q);
      q = fma4(eD, sub4(pc, lds4(row + SRR)), q);
      if (hU) q = fma4(ldg4(cf + CL::WD * PL - P.pitch), sub4(pc, lds4(row - SRR)), q);
    }
#pragma unroll
    for (int j = 0; j < GID_MAX_PAIRS; j++) {
      if (j < P.ns) {
        const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
        const float* fw = row + dy * SRR + dx;
        const float* bw = row - dy * SRR - dx;
        q = fma4(ldg4(cf + (CL::CW + j) * PL), sub4(pc, f4v(fw[0], fw[1], fw[2], fw[3])), q);
        q = fma4(ldg4(cf + (CL::CW + P.ns + j) * PL), sub4(pc, f4v(bw[0], bw[1], bw[2], bw[3])), q);
      }
    }
    finish(c, pc, mul4(q, valid));
  }
  // monochrome block: M_c = w_m sum_k dm_kc p_Tk
  F4 Mc[3];
#pragma unroll
  for (int c = 0; c < 3; c++) Mc[c] = f4s(0.f);
#pragma unroll
  for (int k = 0; k <= K; k++) {
    const F4 pk = lds4(st + k * STC);
#pragma unroll
    for (int c = 0; c < 3; c++) Mc[c] = fma4(f4s(ct.dm[k][c]), pk, Mc[c]);
  }
  {
    const F4 wm = ldg4(cf + CL::WM * PL);
#pragma unroll
    for (int c = 0; c < 3; c++) Mc[c] = mul4(wm, Mc[c]);
  }
  // layers: data and monochrome back-projections, diagonal IRLS weights, smoothness
#pragma unroll 1
  for (int k = 0; k <= K; k++) {
    const float* row = st + k * STC;
    const F4 pk = lds4(row);
    const F4 sR = ldg4(cf + (CL::ER + k) * PL), sD = ldg4(cf + (CL::ED + k) * PL);
    float sLm;
    if constexpr (SHFL) {
      const float sh = __shfl_up_sync(0xffffffffu, sR.b.y, 1);
      sLm = left_lane ? sh : (hL ? cf[(CL::ER + k) * PL - 1] : 0.f);
    } else {
      sLm = hL ? cf[(CL::ER + k) * PL - 1] : 0.f;
    }
    const F4 sL = f4v(sLm, sR.a.x, sR.a.y, sR.b.x);
    const F4 sU = hU ? ldg4(cf + (CL::ED + k) * PL - P.pitch) : f4s(0.f);
    const F4 right = f4v(pk.a.y, pk.b.x, pk.b.y, row[4]);
    const F4 left = f4v(row[-1], pk.a.x, pk.a.y, pk.b.x);
    const F4 down = lds4(row + STR), up = lds4(row - STR);
    F4 q = mul4(ldg4(cf + (CL::WT + k) * PL), pk);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      q = fma4(f4s(ct.b[k][c]), u[c], q);
      q = fma4(f4s(ct.dm[k][c]), Mc[c], q);
    }
    q = fma4(sR, sub4(pk, right), q);
    q = fma4(sL, sub4(pk, left), q);
    q = fma4(sD, sub4(pk, down), q);
    q = fma4(sU, sub4(pk, up), q);
    finish(3 + k, pk, mul4(q, valid));
  }
}

// PCG operator step it: p = z + beta p_old (first step: p = z), q = J^T J p
// from the step's coefficient planes, block partials of <p, q>.  The
// stencil is applied to z only: q = J^T J z + beta q_old equals J^T J p since
// J^T J is fixed within a Gauss-Newton step, so only z needs a halo and p_old,
// q_old are read at the thread's own pixels (p and q may be updated in place).
// mode 1 (stage): q = J^T J pin.  Padding columns (W <= x < pitch) of p, q, z
// and of every coefficient plane are zero and stay zero.
// One operator tile (origin x0, y0): stage s, then q = A s (+ beta q_old) and
// p = s (+ beta p_old) on the tile's pixels.  get_beta() is called once the
// staging loads are in (it may wait on a block reduction).  Returns this
// thread's share of <p, q>.  All threads of the block call it.
// 16-byte asynchronous global -> shared copy (L2 only); src_bytes = 0 writes
// zeros and reads nothing.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((unsigned)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Bulk prefetch of bytes [p, p + bytes) into L2 (no registers, no completion
// to wait for); p 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(p), "r"(bytes) : "memory");
}

// The operator tile's compute phase reads every coefficient plane at the
// tile's own pixels: start those rows towards L2, so that their DRAM latency
// overlaps the staging instead of the dependent math.  None of them is written
// by the PCG vector step, so this may run before the grid dependency on it is
// resolved.  (p_old and q_old, written by the previous operator step, are
// mostly still in L2: prefetching them too measured 0.4 % slower.)
template <int K, int TH>
__device__ __forceinline__ void prefetch_tile(const Params& P, int x0, int y0) {
  constexpr int NTH = BX * TH;
  const int nc = coef_planes(K, P.ns);
  const unsigned bytes = 4u * (unsigned)min(VTW, P.pitch - x0);
  for (int i = tid_flat(); i < nc * TH; i += NTH) {
    const int pl = i / TH, y = y0 + (i - pl * TH);
    if (y < P.H) prefetch_l2(P.coef + (long)pl * P.plane + off2(P, y, x0), bytes);
  }
}

// Programmatic dependent launch: wait until the grid this one depends on has
// completed and its writes are visible (a no-op for an ordinary launch), and
// let the next grid in the stream begin launching.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_release() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// With mapR / mapT (tensor maps of the staged vector, boxes [3][TH + 6][136] and
// [K + 1][TH + 2][136]) the tile is staged by TMA; without them (nullptr) by
// per-thread asynchronous copies.
// Staged chunk i of an operator tile (origin x0, y0): its shared address, its
// plane v and the frame position (gy, gx) of its first float.  Chunks run over
// the reflectance channels' rows y0 - 3 .. y0 + TH + 2, then the layers' rows
// y0 - 1 .. y0 + TH, each row in float4 columns x0 - 4 .. x0 + 131.
template <int K, int TH>
struct TileChunks {
  static constexpr int NCH = VRW / 4;  // float4 chunks per staged row
  static constexpr int NR = 3 * (TH + 2 * AHR) * NCH, NTOT = NR + (K + 1) * (TH + 2) * NCH;
  __device__ __forceinline__ static float* at(ApplyTile<K, TH>& t, int x0, int y0, int i, int& gy, int& gx, int& v) {
    if (i < NR) {
      const int c = i / ((TH + 2 * AHR) * NCH), rem = i - c * (TH + 2 * AHR) * NCH, ly = rem / NCH, lc = rem - ly * NCH;
      gy = y0 - AHR + ly;
      gx = x0 - VHX + 4 * lc;
      v = c;
      return &t.pr[c][ly][4 * lc];
    }
    const int j = i - NR, k = j / ((TH + 2) * NCH), rem = j - k * (TH + 2) * NCH, ly = rem / NCH, lc = rem - ly * NCH;
    gy = y0 - 1 + ly;
    gx = x0 - VHX + 4 * lc;
    v = 3 + k;
    return &t.pt[k][ly][4 * lc];
  }
};

// Stage the V planes at sv (tile and halo, zero outside the frame) into t:
// by TMA with mapR / mapT (tensor maps of sv, boxes [3][TH + 6][136] and
// [K + 1][TH + 2][136]), else by per-thread asynchronous copies.  False in every
// thread if the TMA copy did not complete within the bounded wait (ST_TIMEOUT
// is recorded and the copy still in flight gets a second bounded wait); the
// caller then skips the tile's arithmetic and stores.  All threads call; the
// staged tile is visible to the whole block on return.
template <int K, int TH>
__device__ __forceinline__ bool stage_tile(const Params& P, ApplyTile<K, TH>& t, int x0, int y0,
                                           const float* __restrict__ sv, const CUtensorMap* mapR,
                                           const CUtensorMap* mapT) {
  using TC = TileChunks<K, TH>;
  constexpr int NTH = BX * TH;  // threads per block
  const int tid = tid_flat();
  const bool use_tma = mapR != nullptr && ((smem_addr(&t.pr[0][0][0]) | smem_addr(&t.pt[0][0][0])) & 127u) == 0u;
  if (use_tma) {
    // two TMA boxes (reflectance channels with a 3-row halo, layers with 1),
    // columns x0 - 4 .. x0 + 131 (x0 - 4 is a multiple of 4 floats, also when
    // negative); outside the frame they read as zero
    __shared__ __align__(8) uint64_t bar;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
      mbar_expect_tx(&bar, (unsigned)(sizeof(t.pr) + sizeof(t.pt)));
      tma_load_3d(&t.pr[0][0][0], mapR, x0 - VHX, y0 - AHR, 0, &bar);
      tma_load_3d(&t.pt[0][0][0], mapT, x0 - VHX, y0 - 1, 3, &bar);
    }
    bool done = false;
    for (long i = 0; i < TMA_SPINS && !done; i++) done = mbar_try_wait(&bar, 0);
    if (!__syncthreads_and(done)) {
      // the copy did not complete in time: record it and give the copy still
      // in flight into this block's shared memory a second bounded wait (the
      // status makes the next synchronising call fail)
      if (tid == 0) atomicOr(&P.sc->status, ST_TIMEOUT);
      for (long i = 0; i < TMA_SPINS && !done; i++) done = mbar_try_wait(&bar, 0);
      return false;
    }
  } else {
    // Every chunk is an asynchronous 16-byte copy straight into shared memory
    // (zero-filled outside the frame): all of a thread's copies are in flight
    // at once and hold no registers.
    for (int i = tid; i < TC::NTOT; i += NTH) {
      int gy, gx, v;
      float* dst = TC::at(t, x0, y0, i, gy, gx, v);
      const bool ok = gy >= 0 && gy < P.H && gx >= 0 && gx < P.pitch;
      cp_async16(dst, ok ? sv + v * P.plane + off2(P, gy, gx) : sv, ok ? 16 : 0);
    }
    cp_async_wait_all();
  }
  __syncthreads();
  return true;
}

template <int K, int TH, class GB>
__device__ __forceinline__ float apply_tile(const Params& P, ApplyTile<K, TH>& t, const ColorTable<K>& ct, int x0, int y0,
                                            int mode, int first, GB get_beta, const float* pin, float* pout,
                                            float* __restrict__ qout, const CUtensorMap* mapR = nullptr,
                                            const CUtensorMap* mapT = nullptr) {
  // Stage s = z (PCG step) or s = pin (stage call) with its halo.
  if (!stage_tile<K, TH>(P, t, x0, y0, mode == 0 ? P.z : pin, mapR, mapT)) return 0.f;
  const float beta = get_beta();
  float pq = 0.f;
  const int y = y0 + threadIdx.y, x = x0 + QW * threadIdx.x;
  if (x < P.W && y < P.H) {
    const long o = off2(P, y, x);
    const long PL = P.plane;
    // q = A s on the valid pixels; in a PCG step p = z + beta p_old and, A being
    // fixed within the Gauss-Newton step, q = A p = A z + beta q_old.
    const F4 bb = f4s(beta);
    // Lanes past the frame's right edge: their coefficients are zero and the
    // staged tile reads zero outside the frame, so q and p stay zero there (the
    // first step of every Gauss-Newton step rewrites them from z, whose padding
    // k_linearize has just zeroed).
    auto finish = [&](int v, F4 s, F4 q) {
      F4 p = s;
      const long ov = v * PL + o;
      if (mode == 0 && !first) {
        p = fma4(bb, ldg4(pin + ov), s);
        q = fma4(bb, ldg4(qout + ov), q);
      }
      *reinterpret_cast<float4*>(qout + ov) = to4(q);
      if (mode == 0) *reinterpret_cast<float4*>(pout + ov) = to4(p);
      pq += dot4(p, q);
    };
    const int cx = VHX + QW * threadIdx.x, ry = threadIdx.y + AHR, ty = threadIdx.y + 1;
    op_apply4<K>(P, ct, x, y, &t.pr[0][ry][cx], (TH + 2 * AHR) * VRW, VRW, &t.pt[0][ty][cx], (TH + 2) * VRW,
                           VRW, finish);
  }
  return pq;
}

template <int K, int TH>
__global__ void __launch_bounds__(BX * TH) __maxnreg__(ApplyShape<TH>::MAXREG)
    k_apply(Params P, int mode, int first, int it, int nb_prev, const float* pin, float* pout,
            float* __restrict__ qout, const __grid_constant__ CUtensorMap mapR,
            const __grid_constant__ CUtensorMap mapT) {
  extern __shared__ __align__(128) float4 apply_smem[];
  ApplyTile<K, TH>& t = *reinterpret_cast<ApplyTile<K, TH>*>(apply_smem);
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  prefetch_tile<K, TH>(P, blockIdx.x * VTW, blockIdx.y * TH);
  // everything below reads what the previous PCG vector step wrote
  grid_dep_wait();
  grid_dep_release();
  const bool use_beta = mode == 0 && !first;
  // this thread's share of rho_it = <r, z> from the previous vector step's partials
  const double rho_share = use_beta ? part_share(pcg_partials(P, PART_RZ, it - 1), nb_prev) : 0.0;
  // beta = rho_it / rho_(it-1); block (0, 0) records rho_it for the vector step
  auto get_beta = [&]() -> float {
    if (!use_beta) return 0.f;
    const double rho = block_total(rho_share), rho_old = P.sc->rho2[(it - 1) & 1];
    if (tid_flat() == 0 && blockIdx.x == 0 && blockIdx.y == 0) P.sc->rho2[it & 1] = rho;
    return rho_old != 0.0 ? (float)(rho / rho_old) : 0.f;
  };
  const float pq = apply_tile<K, TH>(P, t, ct, blockIdx.x * VTW, blockIdx.y * TH, mode, first, get_beta, pin, pout, qout,
                                     &mapR, &mapT);
  if (mode != 0) return;
  const double bs = block_sum_f(pq);
  if (tid_flat() == 0) pcg_partials(P, PART_PQ, it)[blockIdx.y * gridDim.x + blockIdx.x] = bs;
}

// ---------------------------------------------------------------- PCG vector step

// PCG vector step it: alpha = rho / <p, q>; delta += alpha p, z -= alpha M^-1 q
// (the residual r = z / M^-1 is never stored), block partials of rho' = <r, z>.
// last 1: X += delta + alpha p (the Gauss-Newton update); last 2: write delta
// only.  Works on whole pitched planes as float4 (the padding columns of every
// PCG vector are zero and stay zero).  A grid of a few blocks per SM strides
// over all V x plane / 4 float4 items, UF items per thread in flight, so that
// only a few hundred blocks pay for the block reduction and the grid fence.
template <int K>
__device__ __forceinline__ float update_range(const Params& P, const float* __restrict__ p, float alpha, int last,
                                              long start, long stride) {
  constexpr int V = K + 4, UF = 2;
  const long n4 = P.plane >> 2, total = (long)V * n4;
  const float4* __restrict__ p4 = reinterpret_cast<const float4*>(p);
  float4* __restrict__ d4 = reinterpret_cast<float4*>(P.d);
  float4* __restrict__ z4 = reinterpret_cast<float4*>(P.z);
  float4* __restrict__ X4 = reinterpret_cast<float4*>(P.X);
  const float4* __restrict__ q4 = reinterpret_cast<const float4*>(P.q);
  const float4* __restrict__ m4 = reinterpret_cast<const float4*>(P.Minv);
  float rz = 0.f;
  auto axpy = [](float a, float4 x, float4 y) {
    return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
  };
  for (long base = start; base < total; base += UF * stride) {
    if (last == 1) {
#pragma unroll
      for (int u = 0; u < UF; u++) {
        const long o = base + u * stride;
        if (o < total) {
          const float4 dn = axpy(alpha, p4[o], d4[o]);
          const float4 xv = X4[o];
          X4[o] = make_float4(xv.x + dn.x, xv.y + dn.y, xv.z + dn.z, xv.w + dn.w);
        }
      }
    } else if (last == 2) {
#pragma unroll
      for (int u = 0; u < UF; u++) {
        const long o = base + u * stride;
        if (o < total) d4[o] = axpy(alpha, p4[o], d4[o]);
      }
    } else {
      // The residual r is not stored: z = M^-1 r is updated directly,
      // z' = z - alpha M^-1 q (= M^-1 (r - alpha q)), and rho' = <r', z'> =
      // sum z'^2 / M^-1.  delta and M^-1 are touched only here: stream them past
      // L2 (evict first) so that z, p, q and the coefficient planes stay resident.
      float4 pv[UF], dv[UF], qv[UF], zv[UF], mv[UF];
#pragma unroll
      for (int u = 0; u < UF; u++) {
        const long o = base + u * stride;
        if (o < total) {
          pv[u] = p4[o];
          dv[u] = __ldcs(d4 + o);
          qv[u] = q4[o];
          zv[u] = z4[o];
          mv[u] = __ldcs(m4 + o);
        }
      }
#pragma unroll
      for (int u = 0; u < UF; u++) {
        const long o = base + u * stride;
        if (o < total) {
          __stcs(d4 + o, axpy(alpha, pv[u], dv[u]));
          const float4 m = mv[u], q = qv[u], z = zv[u];
          const float4 zn = make_float4(fmaf(-alpha, m.x * q.x, z.x), fmaf(-alpha, m.y * q.y, z.y),
                                        fmaf(-alpha, m.z * q.z, z.z), fmaf(-alpha, m.w * q.w, z.w));
          z4[o] = zn;
          // padding entries have M^-1 = 0 and z = 0: they add nothing
          rz += (m.x > 0.f ? zn.x * zn.x / m.x : 0.f) + (m.y > 0.f ? zn.y * zn.y / m.y : 0.f) +
                (m.z > 0.f ? zn.z * zn.z / m.z : 0.f) + (m.w > 0.f ? zn.w * zn.w / m.w : 0.f);
        }
      }
    }
  }
  return rz;
}

// PCG vector step it: alpha = rho / <p, q>; delta += alpha p, z -= alpha M^-1 q,
// block partials of rho' = <r, z> = sum z^2 / M^-1.  last 1: X += delta + alpha p
// (the Gauss-Newton update); last 2: write delta only.  Works on whole pitched
// planes as float4 (the padding columns of every PCG vector are zero and stay
// zero).  A grid of two blocks per SM strides over all V x plane / 4 float4
// items; a 64-register cap for four blocks per SM spilled and measured 10 %
// slower.
template <int K>
__global__ void __launch_bounds__(256, 2) k_update(Params P, int it, int nb_prev, const float* __restrict__ p, int last) {
  grid_dep_wait();  // the operator step's p, q and partials
  grid_dep_release();
  // alpha = rho_it / <p, q>_it from the operator step's partials
  const double pq = block_total(part_share(pcg_partials(P, PART_PQ, it), nb_prev));
  const float alpha = pq != 0.0 ? (float)(P.sc->rho2[it & 1] / pq) : 0.f;
  const float rz = update_range<K>(P, p, alpha, last, (long)blockIdx.x * blockDim.x + threadIdx.x,
                                   (long)gridDim.x * blockDim.x);
  if (last) return;
  const double bs = block_sum_f(rz);
  if (threadIdx.x == 0) pcg_partials(P, PART_RZ, it)[blockIdx.x] = bs;
}

// ---------------------------------------------------------------- work-list PCG steps of a batch

// One video of a work-list launch: the PCG steps of every video of a batch
// that shares K run as one operator launch over all their tiles and one vector
// launch over all their planes, so that small videos do not pay a launch and a
// barely filled wave each, and large ones no wave tail.  Each video keeps its
// own scalars and block partials (its own Params); a block finds its video
// from its index.  Device memory, written by the host when the batch's graph
// is captured.
struct MultiVideo {
  Params P;
  const float* p;  // the video's PCG direction p (updated in place)
  int ntx;         // operator tiles per row
  int ntiles;      // operator tiles
  int nupd;        // vector-step blocks
  int tile0, upd0; // the video's first block in the operator / vector launch
};

// The video (index into vids) that owns block b of a launch (default: this
// block), by first[v] = tile0 or upd0, copied into shared memory; returns the
// block's index within its video.  All threads call.
template <bool UPD>
__device__ __forceinline__ int multi_video(const MultiVideo* __restrict__ vids, int nv, MultiVideo& mv, int& v,
                                           int b = -1) {
  __shared__ int vsel;
  const int tid = tid_flat(), nth = blockDim.x * blockDim.y;
  if (b < 0) b = blockIdx.x;
  if (tid == 0) {
    int s = 0;
    while (s + 1 < nv && (UPD ? vids[s + 1].upd0 : vids[s + 1].tile0) <= b) s++;
    vsel = s;
  }
  __syncthreads();
  v = vsel;
  const int* src = reinterpret_cast<const int*>(vids + v);
  int* dst = reinterpret_cast<int*>(&mv);
  for (int i = tid; i < (int)(sizeof(MultiVideo) / sizeof(int)); i += nth) dst[i] = src[i];
  __syncthreads();
  return b - (UPD ? mv.upd0 : mv.tile0);
}

// Operator step `it` of every video in vids (the work of k_apply, mode 0): block
// b works on tile b - tile0 of its video, with that video's tensor maps
// maps[2 v], maps[2 v + 1] (global memory) and its vector step's nupd partials.
template <int K, int TH>
__global__ void __launch_bounds__(BX * TH) __maxnreg__(ApplyShape<TH>::MAXREG)
    k_apply_multi(const MultiVideo* __restrict__ vids, int nv, const CUtensorMap* __restrict__ maps, int first,
                  int it) {
  extern __shared__ __align__(128) float4 apply_smem[];
  ApplyTile<K, TH>& t = *reinterpret_cast<ApplyTile<K, TH>*>(apply_smem);
  __shared__ ColorTable<K> ct;
  __shared__ MultiVideo mv;
  int v;
  const int local = multi_video<false>(vids, nv, mv, v);
  const Params& P = mv.P;
  load_colors<K>(ct, P.col);
  const int x0 = (local % mv.ntx) * VTW, y0 = (local / mv.ntx) * TH;
  prefetch_tile<K, TH>(P, x0, y0);
  const double rho_share = first ? 0.0 : part_share(pcg_partials(P, PART_RZ, it - 1), mv.nupd);
  auto get_beta = [&]() -> float {
    if (first) return 0.f;
    const double rho = block_total(rho_share), rho_old = P.sc->rho2[(it - 1) & 1];
    if (tid_flat() == 0 && local == 0) P.sc->rho2[it & 1] = rho;
    return rho_old != 0.0 ? (float)(rho / rho_old) : 0.f;
  };
  float* p = const_cast<float*>(mv.p);
  const float pq = apply_tile<K, TH>(P, t, ct, x0, y0, 0, first, get_beta, p, p, P.q, maps + 2 * v, maps + 2 * v + 1);
  const double bs = block_sum_f(pq);
  if (tid_flat() == 0) pcg_partials(P, PART_PQ, it)[local] = bs;
}

// Vector step `it` of every video in vids (the work of k_update): block b is
// block b - upd0 of its video's nupd blocks.
template <int K>
__global__ void __launch_bounds__(256, 2) k_update_multi(const MultiVideo* __restrict__ vids, int nv, int it, int last) {
  __shared__ MultiVideo mv;
  int v;
  const int local = multi_video<true>(vids, nv, mv, v);
  const Params& P = mv.P;
  const double pq = block_total(part_share(pcg_partials(P, PART_PQ, it), mv.ntiles));
  const float alpha = pq != 0.0 ? (float)(P.sc->rho2[it & 1] / pq) : 0.f;
  const float rz =
      update_range<K>(P, mv.p, alpha, last, (long)local * blockDim.x + threadIdx.x, (long)mv.nupd * blockDim.x);
  if (last) return;
  const double bs = block_sum_f(rz);
  if (threadIdx.x == 0) pcg_partials(P, PART_RZ, it)[local] = bs;
}

// ---------------------------------------------------------------- block-Jacobi preconditioner

// Sec. 6.1 names no preconditioner.  Besides the Jacobi default this file offers
// the per-pixel block-Jacobi one: M = blockdiag_x B(x), B(x) the V x V diagonal
// block of J^T J at pixel x.  Only the rows that touch several unknowns of one
// pixel put entries off its diagonal: the three data rows (r_c with every T_k,
// T_k with T_l) and the three monochrome rows (T_k with T_l); every other term
// adds to the diagonal alone.  Variables in plane order r_0..r_2, T_0..T_K;
// a packed lower triangle holds entry (i, j), j <= i, at i (i + 1) / 2 + j.
__host__ __device__ constexpr int tri(int i, int j) { return i * (i + 1) / 2 + j; }

// In-register Cholesky B = L L^T of a packed SPD block; false if a pivot is
// not positive (a block that rounding made indefinite).
template <int V>
__device__ __forceinline__ bool block_cholesky(float (&L)[V * (V + 1) / 2]) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < V; j++) {
    float s = L[tri(j, j)];
#pragma unroll
    for (int k = 0; k < j; k++) s = fmaf(-L[tri(j, k)], L[tri(j, k)], s);
    ok = ok && s > 0.f;
    const float ljj = sqrtf(fmaxf(s, 1e-30f)), inv = 1.0f / ljj;
    L[tri(j, j)] = ljj;
#pragma unroll
    for (int i = j + 1; i < V; i++) {
      float t = L[tri(i, j)];
#pragma unroll
      for (int k = 0; k < j; k++) t = fmaf(-L[tri(i, k)], L[tri(j, k)], t);
      L[tri(i, j)] = t * inv;
    }
  }
  return ok;
}

// y = (L L^T)^-1 r by forward and back substitution (r and y may be one array).
template <int V>
__device__ __forceinline__ void block_solve(const float (&L)[V * (V + 1) / 2], const float (&r)[V], float (&y)[V]) {
#pragma unroll
  for (int i = 0; i < V; i++) {
    float t = r[i];
#pragma unroll
    for (int k = 0; k < i; k++) t = fmaf(-L[tri(i, k)], y[k], t);
    y[i] = t / L[tri(i, i)];
  }
#pragma unroll
  for (int i = V - 1; i >= 0; i--) {
    float t = y[i];
#pragma unroll
    for (int k = i + 1; k < V; k++) t = fmaf(-L[tri(k, i)], y[k], t);
    y[i] = t / L[tri(i, i)];
  }
}

// |L^T z|^2 = z^T B z.
template <int V>
__device__ __forceinline__ float block_norm2(const float (&L)[V * (V + 1) / 2], const float (&z)[V]) {
  float s = 0.f;
#pragma unroll
  for (int j = 0; j < V; j++) {
    float t = 0.f;
#pragma unroll
    for (int i = j; i < V; i++) t = fmaf(L[tri(i, j)], z[i], t);
    s = fmaf(t, t, s);
  }
  return s;
}

// The reflectance part D_r of every block is diagonal (no row couples two
// reflectance channels of a pixel), and its coupling to the layers is
// E[c][k] = l_data R_c^2 S_c b_kc = e_c b_kc.  So a block is kept in Schur form:
//   planes 0..2   1 / D_r,c
//   planes 3..5   e_c
//   planes 6..    the packed Cholesky factor of S = B_T - E^T D_r^-1 E
//                 ((K + 1) x (K + 2) / 2 planes)
// and B y = q is solved as y_T = S^-1 (q_T - E^T D_r^-1 q_r),
// y_r = D_r^-1 (q_r - E y_T); z^T B z = sum_c D_r,c (z_rc + (D_r^-1 E z_T)_c)^2
// + |L_S^T z_T|^2.  6 + (K + 1)(K + 2)/2 planes (34 at K = 6) instead of the
// full factor's (K + 4)(K + 5)/2 (55).
__host__ __device__ constexpr int block_planes(int K) { return 6 + (K + 1) * (K + 2) / 2; }

template <int K>
struct SchurBlock {
  static constexpr int T = K + 1, NS = T * (T + 1) / 2;
  float dinv[3], e[3], L[NS];
};

template <int K>
__device__ __forceinline__ void schur_solve(const SchurBlock<K>& B, const ColorTable<K>& ct, const float (&q)[K + 4],
                                            float (&y)[K + 4]) {
  constexpr int T = K + 1;
  float t[3], r[T];
#pragma unroll
  for (int c = 0; c < 3; c++) t[c] = B.e[c] * B.dinv[c] * q[c];
#pragma unroll
  for (int k = 0; k < T; k++) {
    float v = q[3 + k];
#pragma unroll
    for (int c = 0; c < 3; c++) v = fmaf(-ct.b[k][c], t[c], v);
    r[k] = v;
  }
  float yt[T];
  block_solve<T>(B.L, r, yt);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float ez = 0.f;
#pragma unroll
    for (int k = 0; k < T; k++) ez = fmaf(ct.b[k][c], yt[k], ez);
    y[c] = B.dinv[c] * fmaf(-B.e[c], ez, q[c]);
  }
#pragma unroll
  for (int k = 0; k < T; k++) y[3 + k] = yt[k];
}

template <int K>
__device__ __forceinline__ float schur_norm2(const SchurBlock<K>& B, const ColorTable<K>& ct, const float (&z)[K + 4]) {
  constexpr int T = K + 1;
  float zt[T];
#pragma unroll
  for (int k = 0; k < T; k++) zt[k] = z[3 + k];
  float s = block_norm2<T>(B.L, zt);
#pragma unroll
  for (int c = 0; c < 3; c++) {
    float ez = 0.f;
#pragma unroll
    for (int k = 0; k < T; k++) ez = fmaf(ct.b[k][c], zt[k], ez);
    const float w = fmaf(B.dinv[c] * B.e[c], ez, z[c]);
    s = fmaf(w * w, 1.0f / B.dinv[c], s);
  }
  return s;
}

// Block-Jacobi PCG start, after k_linearize mode 3 (g in z, diag J^T J in Minv):
// form the Schur block from that diagonal and the step's coefficient planes
// (A_c = l_data R_c^2, S_c, the monochrome weight), factor S, store the block
// (P.blk), z = B^-1 g, rho = <g, z>.
template <int K>
__global__ void __launch_bounds__(NT) k_block_factor(Params P) {
  constexpr int V = K + 4, T = K + 1, NS = T * (T + 1) / 2;
  using CL = CoefLayout<K>;
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float rz = 0.f;
  if (x < P.W && y < P.H) {
    const long o = off2(P, y, x);
    const float* cf = P.coef + o;
    float A[3], S[3], dg[V], g[V];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      A[c] = cf[(CL::A + c) * P.plane];
      S[c] = cf[(CL::S + c) * P.plane];
    }
    const float wm = cf[CL::WM * P.plane];
#pragma unroll
    for (int v = 0; v < V; v++) {
      dg[v] = P.Minv[v * P.plane + o];
      g[v] = P.z[v * P.plane + o];
    }
    SchurBlock<K> B;
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      ok = ok && dg[c] > 0.f;
      B.dinv[c] = 1.0f / dg[c];
      B.e[c] = A[c] * S[c];
    }
#pragma unroll
    for (int k = 0; k < T; k++)
#pragma unroll
      for (int l = 0; l <= k; l++) {
        float bt = 0.f, m = 0.f, ee = 0.f;
#pragma unroll
        for (int c = 0; c < 3; c++) {
          bt = fmaf(A[c] * ct.b[k][c], ct.b[l][c], bt);
          m = fmaf(ct.dm[k][c], ct.dm[l][c], m);
          ee = fmaf(B.e[c] * B.e[c] * B.dinv[c] * ct.b[k][c], ct.b[l][c], ee);
        }
        B.L[tri(k, l)] = (l == k ? dg[3 + k] : fmaf(wm, m, bt)) - ee;
      }
    ok = ok && block_cholesky<T>(B.L);
    if (!ok) {  // Jacobi for this pixel
#pragma unroll
      for (int c = 0; c < 3; c++) {
        B.dinv[c] = 1.0f / dg[c];
        B.e[c] = 0.f;
      }
#pragma unroll
      for (int k = 0; k < T; k++)
#pragma unroll
        for (int l = 0; l <= k; l++) B.L[tri(k, l)] = l == k ? sqrtf(dg[3 + k]) : 0.f;
    }
    float* blk = P.blk + o;
#pragma unroll
    for (int c = 0; c < 3; c++) {
      blk[c * P.plane] = B.dinv[c];
      blk[(3 + c) * P.plane] = B.e[c];
    }
#pragma unroll
    for (int j = 0; j < NS; j++) blk[(6 + j) * P.plane] = B.L[j];
    float z[V];
    schur_solve<K>(B, ct, g, z);
#pragma unroll
    for (int v = 0; v < V; v++) {
      P.z[v * P.plane + o] = z[v];
      rz = fmaf(g[v], z[v], rz);
    }
  }
  const double bs = block_sum_f(rz);
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid_flat() == 0) P.partial[b] = bs;
  if (last_block(&P.sc->cnt[CNT_LIN])) {
    const double t = grid_total(P.partial, nb, 1, 0);
    if (tid_flat() == 0) {
      P.sc->rho = t;
      P.sc->rho2[1] = t;  // rho of PCG step 1
      P.sc->rho_hist[0] = t;
      P.sc->beta = 0.0;
      P.sc->cnt[CNT_GRID] = 0u;
    }
  }
}

// Block-Jacobi PCG vector step it: alpha = rho / <p, q>; delta += alpha p,
// z -= alpha B^-1 q (= B^-1 (r - alpha q); r is not stored), block partials of
// rho' = <r', z'> = z'^T B z'.  One pixel per thread, grid-strided over the
// pitched plane (padding columns skipped: their entries are zero).  last 1 / 2
// as for k_update (they do not involve the preconditioner).  Every load of a
// pixel is issued before its first store (a cache-hinted store is ordered
// before the loads that follow it); each thread then holds the whole block,
// so above K = 4 the kernel runs one 256-thread block per SM without a
// register cap (a 128-register cap for two blocks spilled and measured 20 %
// slower at K = 6).
template <int K>
__global__ void __launch_bounds__(256, K <= 4 ? 2 : 1)
    k_update_block(Params P, int it, int nb_prev, const float* __restrict__ p, int last) {
  constexpr int V = K + 4, T = K + 1, NS = T * (T + 1) / 2;
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  grid_dep_wait();  // the operator step's p, q and partials
  grid_dep_release();
  const double pq = block_total(part_share(pcg_partials(P, PART_PQ, it), nb_prev));
  const float alpha = pq != 0.0 ? (float)(P.sc->rho2[it & 1] / pq) : 0.f;
  if (last) {
    update_range<K>(P, p, alpha, last, (long)blockIdx.x * blockDim.x + threadIdx.x, (long)gridDim.x * blockDim.x);
    return;
  }
  // The blocks are read once per step and streamed past L2 (evict first), like
  // delta, so that the operator step's planes stay resident.
  const float* __restrict__ blk = P.blk;
  const float* __restrict__ qv = P.q;
  float* __restrict__ dv = P.d;
  float* __restrict__ zv = P.z;
  const long plane = P.plane;
  float rz = 0.f;
  const unsigned pitch = (unsigned)P.pitch, W = (unsigned)P.W;
  for (long o = (long)blockIdx.x * blockDim.x + threadIdx.x; o < plane; o += (long)gridDim.x * blockDim.x) {
    if ((unsigned)o % pitch >= W) continue;
    SchurBlock<K> B;
    float q[V], y[V], pp[V], dd[V], z[V];
#pragma unroll
    for (int c = 0; c < 3; c++) {
      B.dinv[c] = __ldcs(blk + c * plane + o);
      B.e[c] = __ldcs(blk + (3 + c) * plane + o);
    }
#pragma unroll
    for (int jj = 0; jj < NS; jj++) B.L[jj] = __ldcs(blk + (6 + jj) * plane + o);
#pragma unroll
    for (int v = 0; v < V; v++) {
      q[v] = qv[v * plane + o];
      pp[v] = p[v * plane + o];
      dd[v] = __ldcs(dv + v * plane + o);
      z[v] = zv[v * plane + o];
    }
    schur_solve<K>(B, ct, q, y);
#pragma unroll
    for (int v = 0; v < V; v++) {
      z[v] = fmaf(-alpha, y[v], z[v]);
      __stcs(dv + v * plane + o, fmaf(alpha, pp[v], dd[v]));
      zv[v * plane + o] = z[v];
    }
    rz += schur_norm2<K>(B, ct, z);
  }
  const double bs = block_sum_f(rz);
  if (threadIdx.x == 0) pcg_partials(P, PART_RZ, it)[blockIdx.x] = bs;
}

// ---------------------------------------------------------------- persistent PCG

// Grid-wide barrier of a cooperative launch (all blocks co-resident).  Thread 0
// of each block arrives on a counter; the last to arrive resets it and bumps a
// generation word the others wait on.  Every wait is bounded: after GRID_SPINS
// polls (or the injected limit) the block records ST_TIMEOUT and the barrier
// returns false, and the kernel then returns (so it always terminates).  An
// injected phantom participant makes every block's wait run out.
constexpr long GRID_SPINS = 1L << 22;

__device__ __forceinline__ bool grid_sync(DevScalars* sc) {
  __shared__ int ok;
  __syncthreads();
  if (tid_flat() == 0) {
    volatile unsigned int* gen = &sc->cnt[CNT_GEN];
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int n = gridDim.x * gridDim.y + sc->phantom;
    const long long limit = sc->spin_limit > 0 ? sc->spin_limit : GRID_SPINS;
    if (atomicAdd(&sc->cnt[CNT_GRID], 1u) == n - 1) {
      sc->cnt[CNT_GRID] = 0u;
      __threadfence();
      atomicAdd(&sc->cnt[CNT_GEN], 1u);
      ok = 1;
    } else {
      long long spins = 0;
      while (*gen == g && spins < limit) {
        __nanosleep(64);
        spins++;
      }
      ok = *gen != g;
      if (!ok) atomicOr(&sc->status, ST_TIMEOUT);
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

// All m_inner PCG steps of one Gauss-Newton step in one cooperative launch
// (one block per SM): operator phase (tiles of ATW x TH pixels, grid-strided),
// grid barrier, vector phase (grid-strided float4 items), grid barrier.  Every
// block forms alpha and beta itself from the phase's block partials in the same
// fixed order, so no block waits on a serial reduction and all agree bit for
// bit.  p and q are updated in place.  last_mode as for k_update.
template <int K, int TH>
__global__ void __launch_bounds__(BX * TH) __maxnreg__(ApplyShape<TH>::MAXREG)
    k_pcg(Params P, int m_inner, int last_mode, float* p, float* __restrict__ q) {
  extern __shared__ __align__(128) float4 apply_smem[];
  ApplyTile<K, TH>& t = *reinterpret_cast<ApplyTile<K, TH>*>(apply_smem);
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const int nb = gridDim.x, b = blockIdx.x, tid = tid_flat();
  const int ntx = (P.W + VTW - 1) / VTW, ntiles = ntx * ((P.H + TH - 1) / TH);
  double* part_pq = pcg_partials(P, PART_PQ, 0);
  double* part_rz = pcg_partials(P, PART_RZ, 0);
  double rho = P.sc->rho, rho_old = 0.0;
  for (int m = 1; m <= m_inner; m++) {
    const int first = m == 1;
    const float beta = first ? 0.f : (rho_old != 0.0 ? (float)(rho / rho_old) : 0.f);
    float pq = 0.f;
    for (int tile = b; tile < ntiles; tile += nb) {
      prefetch_tile<K, TH>(P, (tile % ntx) * VTW, (tile / ntx) * TH);
      pq += apply_tile<K, TH>(P, t, ct, (tile % ntx) * VTW, (tile / ntx) * TH, 0, first, [&]() { return beta; }, p, p,
                              q);
      __syncthreads();  // the next tile re-stages shared memory
    }
    double bs = block_sum_f(pq);
    if (tid == 0) part_pq[b] = bs;
    if (!grid_sync(P.sc)) return;
    const double pqs = block_total(part_share(part_pq, nb));
    const float alpha = pqs != 0.0 ? (float)(rho / pqs) : 0.f;
    const int last = m == m_inner ? last_mode : 0;
    const float rz = update_range<K>(P, p, alpha, last, (long)b * blockDim.x * blockDim.y + tid,
                                     (long)nb * blockDim.x * blockDim.y);
    if (last) break;
    bs = block_sum_f(rz);
    if (tid == 0) part_rz[b] = bs;
    if (!grid_sync(P.sc)) return;
    rho_old = rho;
    rho = block_total(part_share(part_rz, nb));
    if (b == 0 && tid == 0 && m < PCG_HIST) P.sc->rho_hist[m] = rho;
  }
}

// The work list of a batch group (videos of one K) as one cooperative launch
// per Gauss-Newton step: all M PCG steps, each an operator phase over the
// group's tiles and a vector phase over its vector blocks of nupd x 256 items
// (both grid-strided over the list, so any number of co-resident blocks covers
// them), separated by bounded grid barriers on the first video's arrival
// counters (cleared by its k_linearize).  Each tile and vector block keeps its
// video's scalars and partial slots exactly as k_apply_multi / k_update_multi
// do.
template <int K, int TH>
__global__ void __launch_bounds__(BX * TH) __maxnreg__(ApplyShape<TH>::MAXREG)
    k_pcg_multi(const MultiVideo* __restrict__ vids, int nv, const CUtensorMap* __restrict__ maps, int ntiles,
                int nupd, int m_inner, DevScalars* bar) {
  extern __shared__ __align__(128) float4 apply_smem[];
  ApplyTile<K, TH>& t = *reinterpret_cast<ApplyTile<K, TH>*>(apply_smem);
  __shared__ ColorTable<K> ct;
  __shared__ MultiVideo mv;
  const int nb = gridDim.x, b = blockIdx.x, tid = tid_flat(), nth = blockDim.x * blockDim.y;
  for (int m = 1; m <= m_inner; m++) {
    const int first = m == 1;
    for (int tile = b; tile < ntiles; tile += nb) {
      int v;
      const int local = multi_video<false>(vids, nv, mv, v, tile);
      const Params& P = mv.P;
      load_colors<K>(ct, P.col);
      const int x0 = (local % mv.ntx) * VTW, y0 = (local / mv.ntx) * TH;
      prefetch_tile<K, TH>(P, x0, y0);
      const double rho_share = first ? 0.0 : part_share(pcg_partials(P, PART_RZ, m - 1), mv.nupd);
      auto get_beta = [&]() -> float {
        if (first) return 0.f;
        const double rho = block_total(rho_share), rho_old = P.sc->rho2[(m - 1) & 1];
        if (tid == 0 && local == 0) P.sc->rho2[m & 1] = rho;
        return rho_old != 0.0 ? (float)(rho / rho_old) : 0.f;
      };
      float* p = const_cast<float*>(mv.p);
      const float pq =
          apply_tile<K, TH>(P, t, ct, x0, y0, 0, first, get_beta, p, p, P.q, maps + 2 * v, maps + 2 * v + 1);
      const double bs = block_sum_f(pq);
      if (tid == 0) pcg_partials(P, PART_PQ, m)[local] = bs;
      __syncthreads();  // the next tile re-stages shared memory and the video record
    }
    if (!grid_sync(bar)) return;
    const int last = m == m_inner ? 1 : 0;
    // vector blocks of 256 items-strides, each done by this block's nth threads
    for (int u = b; u < nupd; u += nb) {
      int v;
      const int local = multi_video<true>(vids, nv, mv, v, u);
      const Params& P = mv.P;
      const double pqs = block_total(part_share(pcg_partials(P, PART_PQ, m), mv.ntiles));
      const float alpha = pqs != 0.0 ? (float)(P.sc->rho2[m & 1] / pqs) : 0.f;
      float rz = 0.f;
      for (int h = tid; h < 256; h += nth)
        rz += update_range<K>(P, mv.p, alpha, last, (long)local * 256 + h, (long)mv.nupd * 256);
      if (!last) {
        const double bs = block_sum_f(rz);
        if (tid == 0) pcg_partials(P, PART_RZ, m)[local] = bs;
      }
      __syncthreads();
    }
    if (last) break;
    if (!grid_sync(bar)) return;
  }
}

// ---------------------------------------------------------------- resident PCG

// All M PCG steps of one Gauss-Newton step in one cooperative launch whose
// blocks keep their share of the PCG state on chip for the whole step, with one
// grid-wide synchronisation per PCG step.  Block b owns one tile of 4 TX x TH
// pixels (tile column b % ntx, tile row b / ntx; thread tid < TX x TH owns the
// four pixels 4 tx .. 4 tx + 3 of the tile's row ty, tx = tid % TX, ty = tid /
// TX) and holds in shared memory
//   ring [RES_NSLOT] slots   coefficient planes of the tile, see below
//   zr  [3][TH + 6][RW]      z of the reflectance channels with a 3-row, 4-column halo
//   zt  [K + 1][TH + 2][RW]  z of the layers with a 1-row, 4-column halo   (RW = 4 TX + 8)
//   ps  [V][TH][4 TX]        p at the tile's pixels
// while M^-1 q (written mq), delta and M^-1 stream from global memory.  The
// operator coefficients stream through the ring: the block's last warp (the
// producer) copies one plane at a time (rows y0 - 1 .. y0 + TH - 1, columns
// x0 - 4 .. x0 + 4 TX + 3: the row above and the column to the left carry the
// up and left edge weights) with TMA into the next free slot, in the order the
// arithmetic consumes them (res_plane), and runs ahead into the next PCG step
// while the block synchronises; every other warp consumes each plane once and
// frees its slot.  PCG step m (z, p, beta and rho = <r, z> known):
//   operator phase: p = z + beta p, q = J^T J z + beta q (the q recurrence of
//     k_apply; q_old = mq_old / M^-1), mq = M^-1 q; block partials of <p, q>,
//     <z, q> and <q, M^-1 q>; the tile's border rows and columns of mq (the
//     part its neighbours' halos need) go to the exchange planes zx;
//   grid all-reduce of the three partials; every block forms alpha = rho /
//     <p, q> and rho' = <r', z'> = rho - 2 alpha <z, q> + alpha^2 <q, M^-1 q>
//     (r' = r - alpha q, z' = z - alpha M^-1 q, and <r, M^-1 q> = <z, q>: the
//     expansion is exact in exact arithmetic), beta' = rho' / rho;
//   vector phase: delta += alpha p, z -= alpha mq on the tile's pixels, and on
//     its halo from the neighbours' published mq, by the same fused
//     multiply-add, so that every block's halo copy stays equal bit for bit to
//     the value its owner holds.
// Textbook PCG needs a second grid-wide step per PCG step (rho' after z'); this
// recurrence needs one.  The operator's arithmetic, in each plane's order, is
// that of op_apply4; the sums differ from the two-kernel loop's in the grouping
// of the FP32 partials and in rho', which is assembled from the three FP64
// totals instead of summed from the updated z.
struct ResTile {
  int TX, TH, ntx, RW;
};

constexpr int RES_NSLOT = 4;    // coefficient ring slots
constexpr int RES_MAXT = 576;   // threads per block at most (18 warps: a register budget of 96)
__host__ __device__ constexpr long res_slot_bytes(int TX, int TH) {
  return ((long)(4 * TX + 8) * (TH + 1) * 4 + 127) / 128 * 128;
}
__host__ __device__ constexpr long res_smem_bytes(int K, int TX, int TH) {
  return 128 + RES_NSLOT * res_slot_bytes(TX, TH) +
         4L * (3L * (TH + 6) * (4 * TX + 8) + (long)(K + 1) * (TH + 2) * (4 * TX + 8) + (long)(K + 4) * TH * (4 * TX));
}
// threads of a resident block: the owners rounded up to whole warps, plus the producer warp
__host__ __device__ constexpr int res_threads(int TX, int TH) { return (TX * TH + 31) / 32 * 32 + 32; }

// Coefficient plane (CoefLayout index) consumed i-th by the resident operator:
// DR, then S_c, A_c for c = 0..2, WR, WD, the consistency pairs (forward,
// backward) j < ns, WM, then WT_k, ER_k, ED_k for k = 0..K.
template <int K>
__device__ __forceinline__ int res_plane(int i, int ns) {
  using CL = CoefLayout<K>;
  if (i == 0) return CL::DR;
  if (i <= 6) return ((i - 1) & 1) ? CL::A + (i - 1) / 2 : CL::S + (i - 1) / 2;
  if (i == 7) return CL::WR;
  if (i == 8) return CL::WD;
  if (i < 9 + 2 * ns) return CL::CW + (((i - 9) & 1) ? ns : 0) + (i - 9) / 2;
  if (i == 9 + 2 * ns) return CL::WM;
  const int r = i - 10 - 2 * ns, k = r / 3, t = r - 3 * k;
  return t == 0 ? CL::WT + k : (t == 1 ? CL::ER + k : CL::ED + k);
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(bar)) : "memory");
}
// bounded wait on an mbarrier phase; false (and ST_TIMEOUT recorded) if it ran out
__device__ __forceinline__ bool mbar_wait_bounded(const Params& P, uint64_t* bar, unsigned parity) {
  for (long i = 0; i < TMA_SPINS; i++)
    if (mbar_try_wait(bar, parity)) return true;
  atomicOr(&P.sc->status, ST_TIMEOUT);
  return false;
}

// q = A s at one thread's four pixels, as op_apply4, with every coefficient
// read from the ring: wait(i) waits for the i-th plane of the sequence and
// returns its slot's element at the thread's first pixel (row stride SW; the
// slot holds the row above and the columns to the left), done(i) frees it.
// The reflectance channels are accumulated side by side, so that each shared
// plane is read once; each channel's operations keep op_apply4's order.
template <int K, class WAIT, class DONE, class FIN>
__device__ __forceinline__ void op_ring4(const Params& P, const ColorTable<K>& ct, int x, const float* sr, int SRC,
                                         int SRR, const float* st, int STC, int STR, int SW, WAIT wait, DONE done,
                                         FIN finish) {
  const F4 valid = f4v(1.f, x + 1 < P.W ? 1.f : 0.f, x + 2 < P.W ? 1.f : 0.f, x + 3 < P.W ? 1.f : 0.f);
  F4 u[3], pc[3], q[3];
#pragma unroll
  for (int c = 0; c < 3; c++) {
    u[c] = f4s(0.f);
    pc[c] = lds4(sr + c * SRC);
  }
#pragma unroll
  for (int k = 0; k <= K; k++) {
    const F4 pk = lds4(st + k * STC);
#pragma unroll
    for (int c = 0; c < 3; c++) u[c] = fma4(f4s(ct.b[k][c]), pk, u[c]);
  }
  int i = 0;
  {  // clustering + temporal diagonal
    const F4 dr = lds4(wait(i));
    done(i++);
#pragma unroll
    for (int c = 0; c < 3; c++) q[c] = mul4(dr, pc[c]);
  }
#pragma unroll
  for (int c = 0; c < 3; c++) {  // data term: u_c = A_c (S_c p_rc + P_c), q_c += S_c u_c
    const F4 Sc = lds4(wait(i));
    done(i++);
    const F4 Ac = lds4(wait(i));
    done(i++);
    u[c] = mul4(Ac, fma4(Sc, pc[c], u[c]));
    q[c] = fma4(Sc, u[c], q[c]);
  }
  {  // r-sparsity: right and left edges, then down and up
    const float* w = wait(i);
    const F4 eR = lds4(w), eL = f4v(w[-1], eR.a.x, eR.a.y, eR.b.x);
    done(i++);
    const float* wd = wait(i);
    const F4 eD = lds4(wd), eU = lds4(wd - SW);
    done(i++);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      const float* row = sr + c * SRC;
      const F4 right = f4v(pc[c].a.y, pc[c].b.x, pc[c].b.y, row[4]);
      const F4 left = f4v(row[-1], pc[c].a.x, pc[c].a.y, pc[c].b.x);
      q[c] = fma4(eR, sub4(pc[c], right), q[c]);
      q[c] = fma4(eL, sub4(pc[c], left), q[c]);
      q[c] = fma4(eD, sub4(pc[c], lds4(row + SRR)), q[c]);
      q[c] = fma4(eU, sub4(pc[c], lds4(row - SRR)), q[c]);
    }
  }
#pragma unroll
  for (int j = 0; j < GID_MAX_PAIRS; j++) {  // consistency pairs (x, x + o_j) and (x - o_j, x)
    if (j < P.ns) {
      const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
      const F4 wf = lds4(wait(i));
      done(i++);
      const F4 wb = lds4(wait(i));
      done(i++);
#pragma unroll
      for (int c = 0; c < 3; c++) {
        const float* fw = sr + c * SRC + dy * SRR + dx;
        const float* bw = sr + c * SRC - dy * SRR - dx;
        q[c] = fma4(wf, sub4(pc[c], f4v(fw[0], fw[1], fw[2], fw[3])), q[c]);
        q[c] = fma4(wb, sub4(pc[c], f4v(bw[0], bw[1], bw[2], bw[3])), q[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < 3; c++) finish(c, pc[c], mul4(q[c], valid));
  // monochrome block: M_c = w_m sum_k dm_kc p_Tk
  F4 Mc[3];
#pragma unroll
  for (int c = 0; c < 3; c++) Mc[c] = f4s(0.f);
#pragma unroll
  for (int k = 0; k <= K; k++) {
    const F4 pk = lds4(st + k * STC);
#pragma unroll
    for (int c = 0; c < 3; c++) Mc[c] = fma4(f4s(ct.dm[k][c]), pk, Mc[c]);
  }
  {
    const F4 wm = lds4(wait(i));
    done(i++);
#pragma unroll
    for (int c = 0; c < 3; c++) Mc[c] = mul4(wm, Mc[c]);
  }
  // layers: diagonal IRLS weights, data and monochrome back-projections, smoothness
#pragma unroll 1
  for (int k = 0; k <= K; k++) {
    const float* row = st + k * STC;
    const F4 pk = lds4(row);
    const F4 wt = lds4(wait(i));
    done(i++);
    const float* er = wait(i);
    const F4 sR = lds4(er), sL = f4v(er[-1], sR.a.x, sR.a.y, sR.b.x);
    done(i++);
    const float* ed = wait(i);
    const F4 sD = lds4(ed), sU = lds4(ed - SW);
    done(i++);
    const F4 right = f4v(pk.a.y, pk.b.x, pk.b.y, row[4]);
    const F4 left = f4v(row[-1], pk.a.x, pk.a.y, pk.b.x);
    const F4 down = lds4(row + STR), up = lds4(row - STR);
    F4 qk = mul4(wt, pk);
#pragma unroll
    for (int c = 0; c < 3; c++) {
      qk = fma4(f4s(ct.b[k][c]), u[c], qk);
      qk = fma4(f4s(ct.dm[k][c]), Mc[c], qk);
    }
    qk = fma4(sR, sub4(pk, right), qk);
    qk = fma4(sL, sub4(pk, left), qk);
    qk = fma4(sD, sub4(pk, down), qk);
    qk = fma4(sU, sub4(pk, up), qk);
    finish(3 + k, pk, mul4(qk, valid));
  }
}

__device__ __forceinline__ unsigned ld_relaxed_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ double* res_slot(const Params& P, unsigned n, int j) {
  return P.xval + ((long)(n % RES_ROWS) * RES_NV + j) * RES_MAXB;
}
__device__ __forceinline__ unsigned* res_count(const Params& P, unsigned n) {
  return reinterpret_cast<unsigned*>(P.xval + (long)RES_ROWS * RES_NV * RES_MAXB) + 32 * (n % RES_ROWS);
}

// Block sums of three per-thread FP32 partials (as block_sum_f, one pass):
// valid in thread 0.
__device__ __forceinline__ void block_sum3_f(float a, float b, float c, double (&out)[RES_NV]) {
  __shared__ float sh[32][RES_NV];
  const int t = tid_flat(), lane = t & 31, wid = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  if (lane == 0) {
    sh[wid][0] = a;
    sh[wid][1] = b;
    sh[wid][2] = c;
  }
  __syncthreads();
  if (wid == 0)
#pragma unroll
    for (int j = 0; j < RES_NV; j++) out[j] = warp_tree(lane < nw ? (double)sh[lane][j] : 0.0);
}

// Grid all-reduce number n (1, 2, ... within the launch) of the resident
// kernel.  part[j] (valid in thread 0) are the block's FP64 partials.  Thread 0
// of block b stores them in its slots of row n % RES_ROWS and adds one to that
// row's arrival counter with release semantics (which also publishes the
// block's earlier global writes: the border mq its neighbours read); it then
// polls the counter (relaxed loads, at most the injected or default poll
// limit) until every block has arrived, and fences.  Every block then reads
// all slots and sums them in the same fixed order, so all blocks hold the same
// totals.  Block 0 clears the counter of row n - 1, which every block has
// finished polling (they all arrived here); it is reused at synchronisation
// n - 1 + RES_ROWS, after the clear is visible to every block (they pass
// synchronisation n + 1 on the way).  The counters start at zero: k_linearize,
// the kernel before every launch, clears them.  False (and ST_TIMEOUT
// recorded) if the wait ran out; all threads of the block agree.
__device__ __forceinline__ bool res_allreduce(const Params& P, unsigned n, const double (&part)[RES_NV],
                                              double (&total)[RES_NV]) {
  const int tid = tid_flat(), nb = gridDim.x;
  bool late = false;
  if (tid == 0) {
#pragma unroll
    for (int j = 0; j < RES_NV; j++) res_slot(P, n, j)[blockIdx.x] = part[j];
    unsigned* cnt = res_count(P, n);
    red_release_add(cnt, 1u);
    const unsigned want = (unsigned)min(nb + (int)P.sc->phantom, RES_MAXB + 1);
    const long long limit = P.sc->spin_limit > 0 ? P.sc->spin_limit : GRID_SPINS;
    bool ok = false;
    for (long long s = 0; s < limit && !ok; s++) ok = ld_relaxed_u32(cnt) >= want;
    late = !ok;
    __threadfence();  // with the polls above: acquires every block's writes
  }
  if (__syncthreads_or(late)) {
    if (tid == 0) atomicOr(&P.sc->status, ST_TIMEOUT);
    return false;
  }
  if (tid == 0 && blockIdx.x == 0 && n > 1) *res_count(P, n - 1) = 0u;
  __shared__ double tot[RES_NV];
  if (tid < 32) {
#pragma unroll
    for (int j = 0; j < RES_NV; j++) {
      const double s = warp_tree(part_share(res_slot(P, n, j), nb));
      if (tid == 0) tot[j] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < RES_NV; j++) total[j] = tot[j];
  return true;
}

template <int K>
__global__ void __launch_bounds__(RES_MAXT, 1)
    k_pcg_resident(Params P, ResTile g, int m_inner, int last_mode, float* __restrict__ mqg,
                   const __grid_constant__ CUtensorMap mapC) {
  constexpr int V = K + 4;
  extern __shared__ __align__(128) float res_smem[];
  __shared__ ColorTable<K> ct;
  __shared__ __align__(8) uint64_t full[RES_NSLOT], empty[RES_NSLOT];
  const int TX = g.TX, TH = g.TH, RW = g.RW, TW = 4 * TX, RR = TH + 6, TR = TH + 2, C4 = RW / 4;
  const int SLOT = (int)(res_slot_bytes(TX, TH) / 4);  // floats per ring slot (row stride RW)
  // the ring's slots are TMA destinations: 128-byte aligned (128 bytes of slack are allocated)
  float* ring = reinterpret_cast<float*>((reinterpret_cast<uintptr_t>(res_smem) + 127) & ~uintptr_t(127));
  float* zr = ring + RES_NSLOT * SLOT;
  float* zt = zr + 3 * RR * RW;
  float* ps = zt + (K + 1) * TR * RW;
  load_colors<K>(ct, P.col);
  const int tid = threadIdx.x, nth = blockDim.x, tx = tid % TX, ty = tid / TX;
  const int nown = (TX * TH + 31) / 32;  // consumer warps; warp nown is the producer
  const bool producer = tid == nown * 32;
  const int x0 = (blockIdx.x % g.ntx) * TW, y0 = (blockIdx.x / g.ntx) * TH;
  const int x = x0 + 4 * tx, y = y0 + ty;
  const bool consumer = tid < nown * 32;
  const bool own = ty < TH && x < P.W && y < P.H;
  const long PL = P.plane, o = own ? off2(P, y, x) : 0;
  const long zxs = (long)V * PL;  // the exchange planes are double-buffered by step parity
  const int NCP = coef_planes(K, P.ns);
  const unsigned box_bytes = (unsigned)((TW + 8) * (TH + 1) * 4);
  if (tid == 0) {
    for (int s = 0; s < RES_NSLOT; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], nown);
    }
  }
  __syncthreads();
  // the producer's copies: sequence plane gi (over the launch) into slot gi % RES_NSLOT
  long issued = 0;
  auto produce = [&](long upto) {
    for (; issued < upto; issued++) {
      const int s = (int)(issued % RES_NSLOT);
      const long use = issued / RES_NSLOT;
      if (use > 0) mbar_wait_bounded(P, &empty[s], (unsigned)((use - 1) & 1));
      mbar_expect_tx(&full[s], box_bytes);
      tma_load_3d(ring + s * SLOT, &mapC, x0 - 4, y0 - 1, res_plane<K>((int)(issued % NCP), P.ns), &full[s]);
    }
  };
  // staged chunk (plane v, staged row ly, float4 column lc): shared address and
  // frame position (gy, gx); in_frame: inside the frame's rows and pitch (the
  // pitch's padding columns are zero in every plane)
  auto chunk = [&](int v, int ly, int lc, int& gy, int& gx) -> float* {
    gy = y0 - (v < 3 ? 3 : 1) + ly;
    gx = x0 - 4 + 4 * lc;
    return v < 3 ? zr + (v * RR + ly) * RW + 4 * lc : zt + ((v - 3) * TR + ly) * RW + 4 * lc;
  };
  auto in_frame = [&](int gy, int gx) { return gy >= 0 && gy < P.H && gx >= 0 && gx < P.pitch; };
  // prologue: the whole staged tile of z from the PCG start; the producer
  // starts the coefficient ring meanwhile
  if (producer) produce(min((long)RES_NSLOT, (long)NCP * m_inner));
  {
    const int nr = 3 * RR * C4, ntot = nr + (K + 1) * TR * C4;
    for (int i = tid; i < ntot; i += nth) {
      int v, r, gy, gx;
      if (i < nr) {
        v = i / (RR * C4);
        r = i - v * RR * C4;
      } else {
        const int k = (i - nr) / (TR * C4);
        v = 3 + k;
        r = i - nr - k * TR * C4;
      }
      float* dst = chunk(v, r / C4, r % C4, gy, gx);
      const bool in = in_frame(gy, gx);
      cp_async16(dst, in ? P.z + v * PL + off2(P, gy, gx) : P.z, in ? 16 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
  }
  // halo chunk i: per reflectance channel the 3 rows above and below (full
  // width) and the 4 columns left and right of the tile's rows; per layer 1 row
  // and the same columns
  const int HR = 6 * C4 + 2 * TH, HT = 2 * C4 + 2 * TH, nhalo = 3 * HR + (K + 1) * HT;
  auto halo = [&](int i, int& v, int& gy, int& gx) -> float* {
    int ly, lc, j;
    if (i < 3 * HR) {
      v = i / HR;
      j = i - v * HR;
      if (j < 6 * C4) {
        const int r = j / C4;
        ly = r < 3 ? r : TH + r;
        lc = j - r * C4;
      } else {
        j -= 6 * C4;
        ly = 3 + (j >> 1);
        lc = (j & 1) ? C4 - 1 : 0;
      }
    } else {
      const int k = (i - 3 * HR) / HT;
      v = 3 + k;
      j = i - 3 * HR - k * HT;
      if (j < 2 * C4) {
        const int r = j / C4;
        ly = r == 0 ? 0 : TH + 1;
        lc = j - r * C4;
      } else {
        j -= 2 * C4;
        ly = 1 + (j >> 1);
        lc = (j & 1) ? C4 - 1 : 0;
      }
    }
    return chunk(v, ly, lc, gy, gx);
  };
  // this thread's chunk is part of a neighbour's halo (reflectance / layers)
  const bool edge_x = tx == 0 || tx == TX - 1;
  const bool pub_r = edge_x || ty < 3 || ty >= TH - 3, pub_t = edge_x || ty == 0 || ty == TH - 1;
  const int oy = own ? ty : 0, ox = own ? tx : 0;  // (threads that own no chunk compute on chunk 0 and discard it)
  float* sr = zr + (oy + 3) * RW + 4 + 4 * ox;
  float* st = zt + (oy + 1) * RW + 4 + 4 * ox;
  float* pp = ps + oy * TW + 4 * ox;
  const int sown = (oy + 1) * RW + 4 + 4 * ox;  // the thread's first pixel in a ring slot
  auto zs = [&](int v) -> float* { return v < 3 ? sr + v * RR * RW : st + (v - 3) * TR * RW; };
  double rho = P.sc->rho;
  float beta = 0.f;
  long consumed = 0;  // ring sequence position of this step's first plane
  for (int m = 1; m <= m_inner; m++) {
    const int first = m == 1;
    float* zx = P.zx + (m & 1) * zxs;
    // operator phase
    float pq = 0.f, zq = 0.f, qmq = 0.f;
    if (consumer) {
      const F4 bb = f4s(beta);
      auto wait = [&](int i) -> const float* {
        const long gi = consumed + i;
        const int s = (int)(gi % RES_NSLOT);
        mbar_wait_bounded(P, &full[s], (unsigned)((gi / RES_NSLOT) & 1));
        return ring + s * SLOT + sown;
      };
      auto done = [&](int i) {
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(&empty[(int)((consumed + i) % RES_NSLOT)]);
      };
      auto finish = [&](int v, F4 s, F4 q) {
        if (!own) return;
        F4 p = s;
        const long ov = v * PL + o;
        float* pv = pp + v * TH * TW;
        const F4 mi = ldc4(P.Minv + ov);
        if (!first) {
          // q_old = mq_old / M^-1 (padding lanes: M^-1 = 0, q_old = 0)
          const float4 mo = __ldcg(reinterpret_cast<const float4*>(mqg + ov));
          const F4 qo = f4v(mi.a.x > 0.f ? __fdividef(mo.x, mi.a.x) : 0.f, mi.a.y > 0.f ? __fdividef(mo.y, mi.a.y) : 0.f,
                            mi.b.x > 0.f ? __fdividef(mo.z, mi.b.x) : 0.f, mi.b.y > 0.f ? __fdividef(mo.w, mi.b.y) : 0.f);
          p = fma4(bb, lds4(pv), s);
          q = fma4(bb, qo, q);
        }
        const F4 mq = mul4(mi, q);
        __stcg(reinterpret_cast<float4*>(mqg + ov), to4(mq));
        if (v < 3 ? pub_r : pub_t) __stcg(reinterpret_cast<float4*>(zx + ov), to4(mq));
        *reinterpret_cast<float4*>(pv) = to4(p);
        pq += dot4(p, q);
        zq += dot4(s, q);
        qmq += dot4(q, mq);
      };
      op_ring4<K>(P, ct, own ? x : 0, sr, RR * RW, RW, st, TR * RW, RW, RW, wait, done, finish);
    } else if (producer) {
      // this step's planes, then the next step's first planes (copied while the
      // block synchronises and runs the vector phase)
      produce(min((long)NCP * m + RES_NSLOT, (long)NCP * m_inner));
    }
    consumed += NCP;
    double part[RES_NV], tot[RES_NV];
    block_sum3_f(pq, zq, qmq, part);
    if (!res_allreduce(P, (unsigned)m, part, tot)) return;
    const double ad = tot[0] != 0.0 ? rho / tot[0] : 0.0;
    const double rho_new = rho - 2.0 * ad * tot[1] + ad * ad * tot[2];
    const float alpha = (float)ad;
    const int last = m == m_inner ? last_mode : 0;
    // vector phase: the halo's loads first, then the tile's pixels, then the halo
    constexpr int HB = 1;
    float4 hmq[HB];
    float* hz[HB];
#pragma unroll
    for (int u = 0; u < HB; u++) {
      hz[u] = nullptr;
      const int i = tid + u * nth;
      if (!last && i < nhalo) {
        int v, gy, gx;
        float* zp = halo(i, v, gy, gx);
        if (in_frame(gy, gx)) {
          hz[u] = zp;
          hmq[u] = __ldcg(reinterpret_cast<const float4*>(zx + v * PL + off2(P, gy, gx)));
        }
      }
    }
    if (own) {
      // all loads of a pair of planes before their stores (a cache-hinted store
      // is ordered before the loads that follow it)
#pragma unroll 1
      for (int v0 = 0; v0 < V; v0 += 2) {
        float4 pv[2], dv[2], mv[2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int v = v0 + u;
          if (v < V) {
            const long ov = v * PL + o;
            pv[u] = *reinterpret_cast<const float4*>(pp + v * TH * TW);
            dv[u] = __ldcg(reinterpret_cast<const float4*>(P.d + ov));
            if (!last) mv[u] = __ldcg(reinterpret_cast<const float4*>(mqg + ov));
          }
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
          const int v = v0 + u;
          if (v >= V) continue;
          const long ov = v * PL + o;
          const float4 p = pv[u], d = dv[u];
          const float4 dn = make_float4(fmaf(alpha, p.x, d.x), fmaf(alpha, p.y, d.y), fmaf(alpha, p.z, d.z),
                                        fmaf(alpha, p.w, d.w));
          if (last == 1) {
            float4* xv = reinterpret_cast<float4*>(P.X + ov);
            const float4 xo = *xv;
            *xv = make_float4(xo.x + dn.x, xo.y + dn.y, xo.z + dn.z, xo.w + dn.w);
            continue;
          }
          __stcg(reinterpret_cast<float4*>(P.d + ov), dn);
          if (last == 2) continue;
          const float4 mq = mv[u];
          float* zp = zs(v);
          const float4 z = *reinterpret_cast<const float4*>(zp);
          *reinterpret_cast<float4*>(zp) = make_float4(fmaf(-alpha, mq.x, z.x), fmaf(-alpha, mq.y, z.y),
                                                       fmaf(-alpha, mq.z, z.z), fmaf(-alpha, mq.w, z.w));
        }
      }
    }
    if (last) break;
    // the halo from the neighbours' published mq, by the owners' operation
#pragma unroll
    for (int u = 0; u < HB; u++) {
      if (hz[u]) {
        const float4 mq = hmq[u], z = *reinterpret_cast<const float4*>(hz[u]);
        *reinterpret_cast<float4*>(hz[u]) = make_float4(fmaf(-alpha, mq.x, z.x), fmaf(-alpha, mq.y, z.y),
                                                        fmaf(-alpha, mq.z, z.z), fmaf(-alpha, mq.w, z.w));
      }
    }
    for (int i = tid + HB * nth; i < nhalo; i += nth) {
      int v, gy, gx;
      float* zp = halo(i, v, gy, gx);
      if (!in_frame(gy, gx)) continue;
      const float4 mq = __ldcg(reinterpret_cast<const float4*>(zx + v * PL + off2(P, gy, gx)));
      const float4 z = *reinterpret_cast<const float4*>(zp);
      *reinterpret_cast<float4*>(zp) = make_float4(fmaf(-alpha, mq.x, z.x), fmaf(-alpha, mq.y, z.y),
                                                   fmaf(-alpha, mq.z, z.z), fmaf(-alpha, mq.w, z.w));
    }
    beta = rho != 0.0 ? (float)(rho_new / rho) : 0.f;
    rho = rho_new;
    if (blockIdx.x == 0 && tid == 0 && m < PCG_HIST) P.sc->rho_hist[m] = rho;
    __syncthreads();
  }
}

// ---------------------------------------------------------------- fused PCG step

// One launch per PCG step (Sec. 6.1's PCG, Jacobi preconditioner), the vector
// step of step it - 1 folded into the operator step it.  Step it - 1 left
// z_(it-1) (buffer zin), mq_(it-1) = M^-1 q_(it-1) (buffer mqin), p_(it-1) and
// the block partials of <p, q>, <z, q>, <q, M^-1 q>.  Every block forms from
// those, in the same fixed order,
//   alpha = rho_(it-1) / <p, q>,
//   rho_it = rho_(it-1) - 2 alpha <z, q> + alpha^2 <q, M^-1 q>   (<r_it, z_it>
//            with r_it = r - alpha q, z_it = z - alpha M^-1 q, expanded),
//   beta = rho_it / rho_(it-1),
// stages z_(it-1) and mq_(it-1) with the stencil's halo (two TMA tiles),
// turns every staged value into z_it = z_(it-1) - alpha mq_(it-1) (the halo's
// owners compute the same values by the same operation), applies A = J^T J to
// it, and at its own pixels forms q_it = A z_it + beta q_(it-1) (q_(it-1) =
// mq_(it-1) / M^-1), p_it = z_it + beta p_(it-1) and delta += alpha p_(it-1),
// writing z_it to zout, M^-1 q_it to mqout, p_it and delta in place.  Step 1
// (it == 1) starts from the PCG start: z_1 = z, p_1 = z, beta = 0, delta
// untouched (zero).  zin / zout and mqin / mqout alternate by step parity:
// neighbouring blocks read the old vectors' halo while this block writes the
// new ones.  The last step's delta += alpha p (and X += delta) is the vector
// step of k_update.  mapR / mapT and mapRq / mapTq: tensor maps of zin and
// mqin.  Where two tiles do not fit in shared memory (MQS false) mq_(it-1) is
// read from global memory, four chunks in flight per thread.
template <int K, int TH>
constexpr bool fused_mq_staged() {
  return 2 * sizeof(ApplyTile<K, TH>) + 4096 <= 227 * 1024;
}

template <int K, int TH>
constexpr size_t fused_smem_bytes() {
  return (fused_mq_staged<K, TH>() ? 2 : 1) * sizeof(ApplyTile<K, TH>);
}

template <int K, int TH>
__global__ void __launch_bounds__(BX * TH) __maxnreg__(ApplyShape<TH>::MAXREG)
    k_pcg_step(Params P, int it, int nb_prev, const float* __restrict__ zin, float* __restrict__ zout,
               const float* __restrict__ mqin, float* __restrict__ mqout, float* __restrict__ p,
               const __grid_constant__ CUtensorMap mapR, const __grid_constant__ CUtensorMap mapT,
               const __grid_constant__ CUtensorMap mapRq, const __grid_constant__ CUtensorMap mapTq) {
  using TC = TileChunks<K, TH>;
  constexpr int NTH = BX * TH;
  constexpr bool MQS = fused_mq_staged<K, TH>();
  extern __shared__ __align__(128) float4 apply_smem[];
  ApplyTile<K, TH>& t = *reinterpret_cast<ApplyTile<K, TH>*>(apply_smem);
  ApplyTile<K, TH>& tq = *(reinterpret_cast<ApplyTile<K, TH>*>(apply_smem) + (MQS ? 1 : 0));
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const int x0 = blockIdx.x * VTW, y0 = blockIdx.y * TH, tid = tid_flat();
  prefetch_tile<K, TH>(P, x0, y0);
  grid_dep_wait();
  grid_dep_release();
  const bool first = it == 1;
  double sh_pq = 0.0, sh_zq = 0.0, sh_qmq = 0.0;
  if (!first) {
    sh_pq = part_share(pcg_partials(P, PART_PQ, it - 1), nb_prev);
    sh_zq = part_share(pcg_partials(P, PART_ZQ, it - 1), nb_prev);
    sh_qmq = part_share(pcg_partials(P, PART_QMQ, it - 1), nb_prev);
  }
  const bool two = MQS && !first;
  if (((smem_addr(&t.pr[0][0][0]) | smem_addr(&t.pt[0][0][0]) | smem_addr(&tq.pr[0][0][0]) |
        smem_addr(&tq.pt[0][0][0])) & 127u) != 0u) {
    // TMA destinations must be 128-byte aligned: per-thread asynchronous copies instead
    for (int i = tid; i < (two ? 2 : 1) * TC::NTOT; i += NTH) {
      int gy, gx, v;
      const bool sec = i >= TC::NTOT;
      float* dst = TC::at(sec ? tq : t, x0, y0, sec ? i - TC::NTOT : i, gy, gx, v);
      const float* src = sec ? mqin : zin;
      const bool ok = gy >= 0 && gy < P.H && gx >= 0 && gx < P.pitch;
      cp_async16(dst, ok ? src + v * P.plane + off2(P, gy, gx) : src, ok ? 16 : 0);
    }
    cp_async_wait_all();
    __syncthreads();
  } else {
    // z_(it-1) and (after step 1, in shared memory) mq_(it-1): one barrier for all boxes
    __shared__ __align__(8) uint64_t bar;
    if (tid == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (tid == 0) {
      mbar_expect_tx(&bar, (unsigned)((two ? 2 : 1) * (sizeof(t.pr) + sizeof(t.pt))));
      tma_load_3d(&t.pr[0][0][0], &mapR, x0 - VHX, y0 - AHR, 0, &bar);
      tma_load_3d(&t.pt[0][0][0], &mapT, x0 - VHX, y0 - 1, 3, &bar);
      if (two) {
        tma_load_3d(&tq.pr[0][0][0], &mapRq, x0 - VHX, y0 - AHR, 0, &bar);
        tma_load_3d(&tq.pt[0][0][0], &mapTq, x0 - VHX, y0 - 1, 3, &bar);
      }
    }
    bool done = false;
    for (long i = 0; i < TMA_SPINS && !done; i++) done = mbar_try_wait(&bar, 0);
    if (!__syncthreads_and(done)) {
      // record the timeout, give the copies still in flight a second bounded
      // wait and write nothing (the status fails the next synchronising call)
      if (tid == 0) atomicOr(&P.sc->status, ST_TIMEOUT);
      for (long i = 0; i < TMA_SPINS && !done; i++) done = mbar_try_wait(&bar, 0);
      return;
    }
  }
  float alpha = 0.f, beta = 0.f;
  if (!first) {
    const double pq = block_total(sh_pq), zq = block_total(sh_zq), qmq = block_total(sh_qmq);
    const double rho = P.sc->rho2[(it - 1) & 1];
    const double ad = pq != 0.0 ? rho / pq : 0.0;
    const double rho_new = rho - 2.0 * ad * zq + ad * ad * qmq;
    alpha = (float)ad;
    beta = rho != 0.0 ? (float)(rho_new / rho) : 0.f;
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
      P.sc->rho2[it & 1] = rho_new;
      if (it - 1 < PCG_HIST) P.sc->rho_hist[it - 1] = rho_new;
    }
    // z_it over the staged tile and halo (outside the frame both tiles read zero)
    auto zstep = [&](float* zs, float4 mq) {
      const float4 z = *reinterpret_cast<const float4*>(zs);
      *reinterpret_cast<float4*>(zs) = make_float4(fmaf(-alpha, mq.x, z.x), fmaf(-alpha, mq.y, z.y),
                                                   fmaf(-alpha, mq.z, z.z), fmaf(-alpha, mq.w, z.w));
    };
    if constexpr (MQS) {
      // the two tiles have one layout: walk both as float4 arrays (padding included)
      float4* zf = reinterpret_cast<float4*>(&t);
      const float4* mf = reinterpret_cast<const float4*>(&tq);
      for (int i = tid; i < (int)(sizeof(ApplyTile<K, TH>) / 16); i += NTH) zstep(reinterpret_cast<float*>(zf + i), mf[i]);
    } else {
      constexpr int U = 4;
      for (int i0 = tid; i0 < TC::NTOT; i0 += U * NTH) {
        float4 mq[U];
        float* zs[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
          int gy, gx, v;
          const int i = i0 + u * NTH;
          zs[u] = nullptr;
          if (i < TC::NTOT) {
            float* a = TC::at(t, x0, y0, i, gy, gx, v);
            if (gy >= 0 && gy < P.H && gx >= 0 && gx < P.pitch) {
              zs[u] = a;
              mq[u] = *reinterpret_cast<const float4*>(mqin + v * P.plane + off2(P, gy, gx));
            }
          }
        }
#pragma unroll
        for (int u = 0; u < U; u++)
          if (zs[u]) zstep(zs[u], mq[u]);
      }
    }
    __syncthreads();
  }
  float pq = 0.f, zq = 0.f, qmq = 0.f;
  const int y = y0 + threadIdx.y, x = x0 + QW * threadIdx.x;
  if (x < P.W && y < P.H) {
    const long o = off2(P, y, x);
    const long PL = P.plane;
    const F4 bb = f4s(beta), aa = f4s(alpha);
    const int cx = VHX + QW * threadIdx.x, ry = threadIdx.y + AHR, ty = threadIdx.y + 1;
    // lanes past the frame's right edge: z, M^-1, p, delta and mq are zero there and stay zero
    auto finish = [&](int v, F4 s, F4 q) {
      const long ov = v * PL + o;
      const F4 mi = ldc4(P.Minv + ov);
      F4 pn = s;
      if (!first) {
        const F4 mo = MQS ? lds4(v < 3 ? &tq.pr[v][ry][cx] : &tq.pt[v - 3][ty][cx]) : ldg4(mqin + ov);
        const F4 qo = f4v(mi.a.x > 0.f ? __fdividef(mo.a.x, mi.a.x) : 0.f, mi.a.y > 0.f ? __fdividef(mo.a.y, mi.a.y) : 0.f,
                          mi.b.x > 0.f ? __fdividef(mo.b.x, mi.b.x) : 0.f, mi.b.y > 0.f ? __fdividef(mo.b.y, mi.b.y) : 0.f);
        const F4 po = ldg4(p + ov);
        pn = fma4(bb, po, s);
        q = fma4(bb, qo, q);
        float4* dv = reinterpret_cast<float4*>(P.d + ov);
        *dv = to4(fma4(aa, po, f4(*dv)));
      }
      const F4 mq = mul4(mi, q);
      *reinterpret_cast<float4*>(zout + ov) = to4(s);
      *reinterpret_cast<float4*>(mqout + ov) = to4(mq);
      *reinterpret_cast<float4*>(p + ov) = to4(pn);
      pq += dot4(pn, q);
      zq += dot4(s, q);
      qmq += dot4(q, mq);
    };
    op_apply4<K>(P, ct, x, y, &t.pr[0][ry][cx], (TH + 2 * AHR) * VRW, VRW, &t.pt[0][ty][cx], (TH + 2) * VRW,
                           VRW, finish);
  }
  double part[RES_NV];
  block_sum3_f(pq, zq, qmq, part);
  if (tid == 0) {
    const int b = blockIdx.y * gridDim.x + blockIdx.x;
    pcg_partials(P, PART_PQ, it)[b] = part[0];
    pcg_partials(P, PART_ZQ, it)[b] = part[1];
    pcg_partials(P, PART_QMQ, it)[b] = part[2];
  }
}

// ---------------------------------------------------------------- base-colour step

// Base-colour refinement (eq:basecolorrefinement): per channel c the K x K
// normal matrix A_c = l_data sum_x R_c^2 T_k T_l + (l_IR + l_CR) I and
// g_c = l_data sum_x R_c T_k e_c, e_c the data residual at the initial colours;
// the last block of each channel solves its SPD system by FP64 Cholesky and
// sets that channel of b = b_init + Delta b.  Grid (nblk, 3): blockIdx.y is the channel; 256
// threads.
// Partials: (K (K + 1) / 2 + K) values x (3 nblk) blocks doubles, value-major.
// VEC: the planes are pitched (pitch a multiple of 4, zero padding) and are
// streamed as float4 by a grid-stride loop; otherwise blocks stride over rows.
template <int K, bool VEC>
__global__ void __launch_bounds__(256) k_dense(Params P, int solve) {
  constexpr int NA = K * (K + 1) / 2, NACC = NA + K, NW = 8;
  __shared__ ColorTable<K> ct;
  __shared__ double wsum[NW][NACC];
  __shared__ double tot[3][NACC];
  load_colors<K>(ct, P.col);
  const int c = blockIdx.y;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; i++) acc[i] = 0.f;
  // one pixel: residual e = I_c - R_c sum_k b_init,kc T_k, a_k = R_c T_k (k >= 1)
  auto pixel = [&](float r, const float* T, float I) {
    const float R = expf(r);
    float S0 = 0.f;
#pragma unroll
    for (int k = 0; k <= K; k++) S0 += ct.bi[k][c] * T[k];
    const float e = I - R * S0;
    float a[K];
#pragma unroll
    for (int k = 0; k < K; k++) a[k] = R * T[k + 1];
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
      for (int l = 0; l <= k; l++) acc[n++] += a[k] * a[l];
#pragma unroll
    for (int k = 0; k < K; k++) acc[NA + k] += a[k] * e;
  };
  if (VEC) {
    // whole pitched planes as float4 (padding columns are zero: r = 0, T = 0, I = 0
    // contribute nothing), a grid-stride loop of one wave
    const long n4 = P.plane >> 2;
    const float4* __restrict__ X4 = reinterpret_cast<const float4*>(P.X);
    const float4* __restrict__ I4 = reinterpret_cast<const float4*>(P.I);
    for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x) {
      const float4 r4 = X4[c * n4 + i], i4 = I4[c * n4 + i];
      float4 t4[K + 1];
#pragma unroll
      for (int k = 0; k <= K; k++) t4[k] = X4[(3 + k) * n4 + i];
      float T[K + 1];
#pragma unroll
      for (int k = 0; k <= K; k++) T[k] = t4[k].x;
      pixel(r4.x, T, i4.x);
#pragma unroll
      for (int k = 0; k <= K; k++) T[k] = t4[k].y;
      pixel(r4.y, T, i4.y);
#pragma unroll
      for (int k = 0; k <= K; k++) T[k] = t4[k].z;
      pixel(r4.z, T, i4.z);
#pragma unroll
      for (int k = 0; k <= K; k++) T[k] = t4[k].w;
      pixel(r4.w, T, i4.w);
    }
  } else {
    for (int y = blockIdx.x; y < P.H; y += gridDim.x)
      for (int x = threadIdx.x; x < P.W; x += blockDim.x) {
        const long o = off2(P, y, x);
        float T[K + 1];
#pragma unroll
        for (int k = 0; k <= K; k++) T[k] = P.X[(3 + k) * P.plane + o];
        pixel(P.X[c * P.plane + o], T, P.I[c * P.plane + o]);
      }
  }
  // block reduction: FP32 warp shuffles, then the 8 warp sums in order
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < NACC; i++) {
    float v = acc[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[wid][i] = (double)v;
  }
  __syncthreads();
  const int nbt = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (threadIdx.x < NACC) {
    double s = 0.0;
    for (int ww = 0; ww < NW; ww++) s += wsum[ww][threadIdx.x];
    P.partial[(long)threadIdx.x * nbt + b] = s;
  }
  // the last block of each channel reduces and solves that channel's system
  if (!last_block(&P.sc->cnt[CNT_DENSE + c], gridDim.x)) return;
  // each warp sums whole value rows: lanes stride the blocks, then a shuffle tree
  for (int i = wid; i < NACC; i += NW) {
    const double* src = P.partial + (long)i * nbt + (long)c * gridDim.x;
    double s = 0.0;
    for (int bb = lane; bb < (int)gridDim.x; bb += 32) s += __ldcg(src + bb);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) tot[c][i] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int cc = c;
    const double ld = P.w.ld, ridge = (double)P.w.lIR + (double)P.w.lCR;
    double A[K][K], L[K][K], g[K], yv[K], xs[K];
    int n = 0;
#pragma unroll
    for (int k = 0; k < K; k++)
#pragma unroll
      for (int l = 0; l <= k; l++) {
        A[k][l] = A[l][k] = ld * tot[cc][n++];
      }
#pragma unroll
    for (int k = 0; k < K; k++) {
      A[k][k] += ridge;
      g[k] = ld * tot[cc][NA + k];
    }
#pragma unroll
    for (int k = 0; k < K; k++) {
      P.sc->g[cc * K + k] = g[k];
#pragma unroll
      for (int l = 0; l < K; l++) P.sc->A[(cc * K + k) * K + l] = A[k][l];
    }
    if (solve) {
      bool ok = true;
      double rd[K];  // 1 / L_jj
#pragma unroll
      for (int j = 0; j < K; j++) {
        double s = A[j][j];
#pragma unroll
        for (int m = 0; m < j; m++) s -= L[j][m] * L[j][m];
        ok = ok && (s > 0.0);
        L[j][j] = sqrt(s > 0.0 ? s : 1.0);
        rd[j] = 1.0 / L[j][j];
#pragma unroll
        for (int i = j + 1; i < K; i++) {
          double tt = A[i][j];
#pragma unroll
          for (int m = 0; m < j; m++) tt -= L[i][m] * L[j][m];
          L[i][j] = tt * rd[j];
        }
      }
      if (ok) {
#pragma unroll
        for (int i = 0; i < K; i++) {
          double tt = g[i];
#pragma unroll
          for (int m = 0; m < i; m++) tt -= L[i][m] * yv[m];
          yv[i] = tt * rd[i];
        }
#pragma unroll
        for (int i = K - 1; i >= 0; i--) {
          double tt = yv[i];
#pragma unroll
          for (int m = i + 1; m < K; m++) tt -= L[m][i] * xs[m];
          xs[i] = tt * rd[i];
        }
#pragma unroll
        for (int k = 0; k < K; k++) {
          const double bn = (double)P.col->binit[k * 3 + cc] + xs[k];
          P.col->bd[k * 3 + cc] = bn;
          P.col->b[k * 3 + cc] = (float)bn;
        }
      } else {
        atomicOr(&P.sc->status, ST_SINGULAR);
      }
    }
  }
}

// Exact energy (eq:giv-energy), 8 FP64 sums into sc->energy; with a mask, the
// terms evaluated at the masked pixels only (each pixel owns its data,
// clustering, monochrome, i-sparsity and non-neg terms and the pair / edge
// terms evaluated at it).
template <int K>
__global__ void __launch_bounds__(NT) k_energy(Params P, const uint8_t* __restrict__ mask) {
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const Weights& w = P.w;
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float E[8];
  for (int i = 0; i < 8; i++) E[i] = 0.f;
  // with a mask (H x W, dense): only the terms evaluated at its nonzero pixels
  if (x < P.W && y < P.H && (!mask || mask[(long)y * P.W + x])) {
    const long o = off2(P, y, x);
    PixState<K> s;
    load_state<K>(P, ct, o, s);
    const int l = P.lab[o];
    const float* bcl = w.rcluster_follows_b ? P.col->b : P.col->binit;
    const float Sbar = (s.S[0] + s.S[1] + s.S[2]) * (1.0f / 3.0f);
    for (int c = 0; c < 3; c++) {
      const float e = P.I[c * P.plane + o] - s.R[c] * s.S[c];
      E[0] += w.ld * e * e;
      const float dcl = s.rr[c] - logf(bcl[l * 3 + c]);
      E[1] += w.lcl * dcl * dcl;
      E[4] += w.lm * P.wsr[o] * (s.S[c] - Sbar) * (s.S[c] - Sbar);
    }
    float g2 = 0.f;
    for (int c = 0; c < 3; c++) {
      if (x + 1 < P.W) {
        float dd = P.X[c * P.plane + o + 1] - s.rr[c];
        g2 += dd * dd;
      }
      if (y + 1 < P.H) {
        float dd = P.X[c * P.plane + o + P.pitch] - s.rr[c];
        g2 += dd * dd;
      }
    }
    E[2] = w.lrs * (w.p == 1.0f ? sqrtf(g2) : powf(sqrtf(g2), w.p));
    for (int j = 0; j < P.ns; j++) {
      const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
      if (!inside(P, y + dy, x + dx)) continue;
      const long n = o + (long)dy * P.pitch + dx;
      float d2 = 0.f;
      for (int c = 0; c < 3; c++) {
        float dd = s.rr[c] - P.X[c * P.plane + n];
        d2 += dd * dd;
      }
      E[3] += w.lrc * P.ws[j * P.plane + o] * d2;
    }
    if (P.temporal)
      for (int j = 0; j < P.nt; j++) {
        const int dy = P.off_t[2 * j], dx = P.off_t[2 * j + 1];
        if (!inside(P, y + dy, x + dx)) continue;
        const long n = o + (long)dy * P.pitch + dx;
        float d2 = 0.f;
        for (int c = 0; c < 3; c++) {
          float dd = s.rr[c] - P.rprev[c * P.plane + n];
          d2 += dd * dd;
        }
        E[3] += w.lrc * P.wt[j * P.plane + o] * d2;
      }
#pragma unroll
    for (int k = 0; k <= K; k++) {
      const float t = s.T[k];
      if (k > 0) E[5] += w.lis * fabsf(t);
      if (x + 1 < P.W) E[6] += w.lsm * fabsf(P.X[(3 + k) * P.plane + o + 1] - t);
      if (y + 1 < P.H) E[6] += w.lsm * fabsf(P.X[(3 + k) * P.plane + o + P.pitch] - t);
      E[7] += w.lnn * fmaxf(-t, 0.f);
    }
  }
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  for (int i = 0; i < 8; i++) {
    const double s = block_sum_f(E[i]);
    if (tid_flat() == 0) P.partial[(long)b * 8 + i] = s;
  }
  if (last_block(&P.sc->cnt[CNT_ENERGY]))
    for (int i = 0; i < 8; i++) {
      const double t = grid_total(P.partial, nb, 8, i);
      if (tid_flat() == 0) P.sc->energy[i] = t;
    }
}

// Read-out: R = exp(r) and T planes to contiguous outputs.
template <int K>
__global__ void k_readout(Params P, float* __restrict__ Rout, float* __restrict__ Tout) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  const long o = off2(P, y, x), HW = (long)P.H * P.W, dst = (long)y * P.W + x;
  if (Rout)
    for (int c = 0; c < 3; c++) Rout[c * HW + dst] = expf(P.X[c * P.plane + o]);
  if (Tout)
    for (int k = 0; k <= K; k++) Tout[k * HW + dst] = P.X[(3 + k) * P.plane + o];
}

// Labels of one correction candidate: region pixels (mask != 0) take label k.
__global__ void k_relabel(const uint8_t* __restrict__ lab, const uint8_t* __restrict__ region, uint8_t k,
                          uint8_t* __restrict__ out, long n) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = region[i] ? k : lab[i];
}

// ---------------------------------------------------------------- editing

// New base colours and per-layer gains of a layer recombination.
struct EditTable {
  float bn[GID_MAX_K * 3];
  float gain[GID_MAX_K];
};

// Layer recombination (Sec. 7.4): I'(x) = R'(x) (T_0 + sum_k g_k b'_k T_k(x)),
// R'_c = R_c b'_jc / b_jc where mask(x) = j in 1..K (the pixel belongs to an
// object of base colour j being recoloured) and b_jc != 0, else R.  b is the
// context's current (refined) colour set.  Planar output, 3 x H x W.
template <int K>
__global__ void k_recombine(Params P, EditTable e, const uint8_t* __restrict__ mask, float* __restrict__ out) {
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  if (x >= P.W || y >= P.H) return;
  const long o = off2(P, y, x), HW = (long)P.H * P.W, dst = (long)y * P.W + x;
  float T[K + 1];
#pragma unroll
  for (int k = 0; k <= K; k++) T[k] = P.X[(3 + k) * P.plane + o];
  int j = mask ? mask[dst] : 0;
  j = j <= K ? j : 0;
  for (int c = 0; c < 3; c++) {
    float S = T[0];
#pragma unroll
    for (int k = 1; k <= K; k++) S += e.gain[k - 1] * e.bn[(k - 1) * 3 + c] * T[k];
    float R = expf(P.X[c * P.plane + o]);
    if (j > 0) {
      const float bo = P.col->b[(j - 1) * 3 + c];
      if (bo != 0.f) R *= e.bn[(j - 1) * 3 + c] / bo;
    }
    out[c * HW + dst] = R * S;
  }
}

}  // namespace gid
