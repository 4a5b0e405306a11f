// Device kernels of the illumination decomposition solver (sm_103a).
//
// Unknowns per pixel (V = K + 4): r_R, r_G, r_B (r = ln R) and T_0..T_K, stored
// as V float32 planes [V][H][pitch] (pitch a multiple of 32 floats, 128-byte
// rows).  One thread owns one pixel in the stencil kernels; blocks are 32 x 8.
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

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gid.h"

namespace gid {

constexpr int BX = 32, BY = 8, NT = BX * BY;

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

enum : int { ST_BAD_LABEL = 1, ST_SINGULAR = 2 };

struct DevScalars {
  double rho, pq, alpha, beta;
  double energy[8];
  double A[3 * GID_MAX_K * GID_MAX_K];
  double g[3 * GID_MAX_K];
  unsigned int cnt[8];
  int status;
};
enum { CNT_LIN, CNT_APPLY, CNT_UPDATE, CNT_DENSE, CNT_ENERGY };

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
  float* r;
  float* z;
  float* q;
  float* Minv;
  DevColors* col;
  DevScalars* sc;
  double* partial;
};

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ int tid_flat() { return threadIdx.y * blockDim.x + threadIdx.x; }

// Sum of v over the block; the result is valid in thread 0.  All threads call.
__device__ __forceinline__ double block_sum(double v) {
  __shared__ double sh[32];
  const int t = tid_flat(), lane = t & 31, wid = t >> 5;
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (wid == 0) {
    s = lane < nw ? sh[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  __syncthreads();
  return s;
}

// True in every thread of the last block to arrive.  Thread 0 must have
// written this block's partials before the call.  Resets the counter.
__device__ __forceinline__ bool last_block(unsigned int* cnt) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (tid_flat() == 0) {
    const unsigned int n = gridDim.x * gridDim.y * gridDim.z;
    const unsigned int t = atomicAdd(cnt, 1u);
    is_last = (t == n - 1);
    if (is_last) *cnt = 0u;
  }
  __syncthreads();
  if (is_last) __threadfence();
  return is_last;
}

// Sum of n partials (stride `stride`, starting at `base`) in a fixed order.
__device__ __forceinline__ double grid_total(const double* partial, int n, int stride, int base) {
  double s = 0.0;
  for (int i = tid_flat(); i < n; i += blockDim.x * blockDim.y) s += __ldcg(partial + (long)i * stride + base);
  return block_sum(s);
}

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
  if (x >= P.W || y >= P.H) return;
  const long o = off2(P, y, x);
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

// q = (J^T J) p at one pixel.  pf(v, dy, dx) returns p at a neighbour (only
// called for in-image neighbours).  pc holds p at the pixel.
template <int K, class PF>
__device__ __forceinline__ void normal_apply(const Params& P, const ColorTable<K>& ct, const Pix& px, long o,
                                             const PixState<K>& s, const float* pc, PF pf, float* qv) {
  constexpr int V = K + 4;
  const Weights& w = P.w;
#pragma unroll
  for (int v = 0; v < V; v++) qv[v] = 0.f;
  // E_data (eq:data-term): rank-3 block of the pixel.
  for (int c = 0; c < 3; c++) {
    float Pc = 0.f;
#pragma unroll
    for (int k = 0; k <= K; k++) Pc += ct.b[k][c] * pc[3 + k];
    const float u = w.ld * s.R[c] * s.R[c] * (s.S[c] * pc[c] + Pc);
    qv[c] += s.S[c] * u;
#pragma unroll
    for (int k = 0; k <= K; k++) qv[3 + k] += ct.b[k][c] * u;
  }
  // E_clustering (eq:clustering-term): diagonal.
  for (int c = 0; c < 3; c++) qv[c] += w.lcl * pc[c];
  // E_r-sparsity (eq:reflectance-sparsity-term): 4-neighbour stencil on r.
  const Edges er = rsparse_edges(P, P.X, px);
  for (int c = 0; c < 3; c++) qv[c] += edge_laplace(er, px, pc[c], [&](int dy, int dx) { return pf(c, dy, dx); });
  // E_r-consistency, spatial pairs (x, x + o_j) and (x - o_j, x).
  for (int j = 0; j < P.ns; j++) {
    const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
    if (inside(P, px.y + dy, px.x + dx)) {
      const float of = w.lrc * P.ws[j * P.plane + o];
      for (int c = 0; c < 3; c++) qv[c] += of * (pc[c] - pf(c, dy, dx));
    }
    if (inside(P, px.y - dy, px.x - dx)) {
      const float ob = w.lrc * P.ws[j * P.plane + o - (long)dy * P.pitch - dx];
      for (int c = 0; c < 3; c++) qv[c] += ob * (pc[c] - pf(c, -dy, -dx));
    }
  }
  // E_r-consistency, temporal pairs: diagonal (the previous frame is fixed).
  if (P.temporal) {
    const float wt = w.lrc * P.wtsum[o];
    for (int c = 0; c < 3; c++) qv[c] += wt * pc[c];
  }
  // E_monochrome (Sec. 5.2): rank-3 block on T.
  const float wm = w.lm * P.wsr[o];
  for (int c = 0; c < 3; c++) {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k <= K; k++) m += ct.dm[k][c] * pc[3 + k];
    m *= wm;
#pragma unroll
    for (int k = 0; k <= K; k++) qv[3 + k] += ct.dm[k][c] * m;
  }
  // E_i-sparsity (k >= 1) and E_non-neg (all k): diagonal IRLS weights.
#pragma unroll
  for (int k = 0; k <= K; k++) {
    float wd = nonneg_weight(w, s.T[k]);
    if (k > 0) wd += irls_l1(w, w.lis, s.T[k]);
    qv[3 + k] += wd * pc[3 + k];
  }
  // E_smoothness (eq:smoothness-term): 4-neighbour stencil per layer.
#pragma unroll
  for (int k = 0; k <= K; k++) {
    const Edges es = smooth_edges(P, P.X, 3 + k, px, s.T[k]);
    qv[3 + k] += edge_laplace(es, px, pc[3 + k], [&](int dy, int dx) { return pf(3 + k, dy, dx); });
  }
}

// Linearisation (fused): g = -J^T F, diag(J^T J); PCG start r = g, z = M^-1 r.
// mode 0: PCG init (writes r, z, Minv, zero delta, rho); mode 1: stage output
// (writes g to gout and diag to dout).
template <int K>
__global__ void __launch_bounds__(NT) k_linearize(Params P, int mode, float* __restrict__ gout,
                                                  float* __restrict__ dout) {
  constexpr int V = K + 4;
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const Weights& w = P.w;
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float rz = 0.f;
  if (x < P.W && y < P.H) {
    const Pix px = make_pix(P, x, y);
    const long o = off2(P, y, x);
    PixState<K> s;
    load_state<K>(P, ct, o, s);
    float g[V], dg[V];
#pragma unroll
    for (int v = 0; v < V; v++) g[v] = dg[v] = 0.f;
    // Linear terms: g -= A_lin X and diag += diag(A_lin), with the same stencil
    // as normal_apply; the data term is handled separately below.
    const float* X = P.X;
    auto xf = [&](int v, int dy, int dx) { return X[v * P.plane + o + (long)dy * P.pitch + dx]; };
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
    const Edges er = rsparse_edges(P, X, px);
    for (int c = 0; c < 3; c++) {
      g[c] -= edge_laplace(er, px, s.rr[c], [&](int dy, int dx) { return xf(c, dy, dx); });
      dg[c] += er.R + er.D + er.L + er.U;
    }
    // E_r-consistency, spatial.
    for (int j = 0; j < P.ns; j++) {
      const int dy = P.off_s[2 * j], dx = P.off_s[2 * j + 1];
      if (inside(P, y + dy, x + dx)) {
        const float of = w.lrc * P.ws[j * P.plane + o];
        for (int c = 0; c < 3; c++) {
          g[c] -= of * (s.rr[c] - xf(c, dy, dx));
          dg[c] += of;
        }
      }
      if (inside(P, y - dy, x - dx)) {
        const float ob = w.lrc * P.ws[j * P.plane + o - (long)dy * P.pitch - dx];
        for (int c = 0; c < 3; c++) {
          g[c] -= ob * (s.rr[c] - xf(c, -dy, -dx));
          dg[c] += ob;
        }
      }
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
#pragma unroll
    for (int k = 0; k <= K; k++) {
      float wd = nonneg_weight(w, s.T[k]);
      if (k > 0) wd += irls_l1(w, w.lis, s.T[k]);
      g[3 + k] -= wd * s.T[k];
      dg[3 + k] += wd;
    }
    // E_smoothness.
#pragma unroll
    for (int k = 0; k <= K; k++) {
      const Edges es = smooth_edges(P, X, 3 + k, px, s.T[k]);
      g[3 + k] -= edge_laplace(es, px, s.T[k], [&](int dy, int dx) { return xf(3 + k, dy, dx); });
      dg[3 + k] += es.R + es.D + es.L + es.U;
    }
    if (mode == 0) {
#pragma unroll
      for (int v = 0; v < V; v++) {
        const long ov = v * P.plane + o;
        const float mi = 1.0f / dg[v];
        const float zz = mi * g[v];
        P.Minv[ov] = mi;
        P.r[ov] = g[v];
        P.z[ov] = zz;
        P.d[ov] = 0.f;
        rz += g[v] * zz;
      }
    } else {
#pragma unroll
      for (int v = 0; v < V; v++) {
        const long ov = v * P.plane + o;
        gout[ov] = g[v];
        dout[ov] = dg[v];
      }
    }
  }
  if (mode != 0) return;
  const double bs = block_sum((double)rz);
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid_flat() == 0) P.partial[b] = bs;
  if (last_block(&P.sc->cnt[CNT_LIN])) {
    const double t = grid_total(P.partial, nb, 1, 0);
    if (tid_flat() == 0) {
      P.sc->rho = t;
      P.sc->beta = 0.0;
    }
  }
}

// PCG operator step: p = z + beta p_old (first step: p = z), q = J^T J p,
// <p, q> reduced, alpha = rho / <p, q>.  mode 1 (stage): p = pin, only q.
template <int K>
__global__ void __launch_bounds__(NT) k_apply(Params P, int mode, int first, const float* __restrict__ pin,
                                              float* __restrict__ pout, float* __restrict__ qout) {
  constexpr int V = K + 4;
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const float beta = (mode == 0 && !first) ? (float)P.sc->beta : 0.f;
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float pq = 0.f;
  if (x < P.W && y < P.H) {
    const Pix px = make_pix(P, x, y);
    const long o = off2(P, y, x);
    const float* __restrict__ z = P.z;
    auto pf = [&](int v, int dy, int dx) -> float {
      const long a = v * P.plane + o + (long)dy * P.pitch + dx;
      if (mode != 0) return pin[a];
      return first ? z[a] : fmaf(beta, pin[a], z[a]);
    };
    PixState<K> s;
    load_state<K>(P, ct, o, s);
    float pc[V], qv[V];
#pragma unroll
    for (int v = 0; v < V; v++) pc[v] = pf(v, 0, 0);
    normal_apply<K>(P, ct, px, o, s, pc, pf, qv);
#pragma unroll
    for (int v = 0; v < V; v++) {
      const long ov = v * P.plane + o;
      qout[ov] = qv[v];
      if (mode == 0) pout[ov] = pc[v];
      pq += pc[v] * qv[v];
    }
  }
  if (mode != 0) return;
  const double bs = block_sum((double)pq);
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid_flat() == 0) P.partial[b] = bs;
  if (last_block(&P.sc->cnt[CNT_APPLY])) {
    const double t = grid_total(P.partial, nb, 1, 0);
    if (tid_flat() == 0) {
      P.sc->pq = t;
      P.sc->alpha = t != 0.0 ? P.sc->rho / t : 0.0;
    }
  }
}

// PCG vector step: delta += alpha p, r -= alpha q, z = M^-1 r, rho' = <r, z>,
// beta = rho' / rho.  last 1: X += delta + alpha p (the Gauss-Newton update);
// last 2: write delta only.
template <int K>
__global__ void __launch_bounds__(NT) k_update(Params P, const float* __restrict__ p, int last) {
  constexpr int V = K + 4;
  const float alpha = (float)P.sc->alpha;
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float rz = 0.f;
  if (x < P.W && y < P.H) {
    const long o = off2(P, y, x);
#pragma unroll
    for (int v = 0; v < V; v++) {
      const long ov = v * P.plane + o;
      const float dn = fmaf(alpha, p[ov], P.d[ov]);
      if (last == 1) {
        P.X[ov] += dn;
      } else if (last == 2) {
        P.d[ov] = dn;
      } else {
        P.d[ov] = dn;
        const float rn = fmaf(-alpha, P.q[ov], P.r[ov]);
        const float zz = P.Minv[ov] * rn;
        P.r[ov] = rn;
        P.z[ov] = zz;
        rz += rn * zz;
      }
    }
  }
  if (last) return;
  const double bs = block_sum((double)rz);
  const int nb = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
  if (tid_flat() == 0) P.partial[b] = bs;
  if (last_block(&P.sc->cnt[CNT_UPDATE])) {
    const double t = grid_total(P.partial, nb, 1, 0);
    if (tid_flat() == 0) {
      const double rho = P.sc->rho;
      P.sc->beta = rho != 0.0 ? t / rho : 0.0;
      P.sc->rho = t;
    }
  }
}

// Base-colour refinement (eq:basecolorrefinement): per channel c the K x K
// normal matrix A_c = l_data sum_x R_c^2 T_k T_l + (l_IR + l_CR) I and
// g_c = l_data sum_x R_c T_k e_c, e_c the data residual at the initial colours;
// the last block solves the three SPD systems by FP64 Cholesky and sets
// b = b_init + Delta b.  Grid (nblk, 3): blockIdx.y is the channel.
template <int K>
__global__ void __launch_bounds__(256) k_dense(Params P, int solve) {
  constexpr int NA = K * (K + 1) / 2, NACC = NA + K;
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const int c = blockIdx.y;
  const long HW = (long)P.H * P.W;
  float acc[NACC];
#pragma unroll
  for (int i = 0; i < NACC; i++) acc[i] = 0.f;
  const long stride = (long)gridDim.x * blockDim.x;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += stride) {
    const int y = (int)(i / P.W), x = (int)(i - (long)y * P.W);
    const long o = off2(P, y, x);
    const float R = expf(P.X[c * P.plane + o]);
    float T[K + 1];
#pragma unroll
    for (int k = 0; k <= K; k++) T[k] = P.X[(3 + k) * P.plane + o];
    float S0 = 0.f;
#pragma unroll
    for (int k = 0; k <= K; k++) S0 += ct.bi[k][c] * T[k];
    const float e = P.I[c * P.plane + o] - R * S0;
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
  }
  const int b = blockIdx.y * gridDim.x + blockIdx.x;
  for (int i = 0; i < NACC; i++) {
    const double s = block_sum((double)acc[i]);
    if (threadIdx.x == 0) P.partial[(long)b * NACC + i] = s;
  }
  if (!last_block(&P.sc->cnt[CNT_DENSE])) return;
  __shared__ double tot[3][NACC];
  for (int cc = 0; cc < 3; cc++)
    for (int i = 0; i < NACC; i++) {
      double s = 0.0;
      for (int bb = threadIdx.x; bb < (int)gridDim.x; bb += blockDim.x)
        s += __ldcg(P.partial + (long)(cc * gridDim.x + bb) * NACC + i);
      s = block_sum(s);
      if (threadIdx.x == 0) tot[cc][i] = s;
    }
  __syncthreads();
  if (threadIdx.x < 3) {
    const int cc = threadIdx.x;
    const double ld = P.w.ld, ridge = (double)P.w.lIR + (double)P.w.lCR;
    double A[K][K], L[K][K], g[K], yv[K], xs[K];
    int n = 0;
    for (int k = 0; k < K; k++)
      for (int l = 0; l <= k; l++) {
        A[k][l] = A[l][k] = ld * tot[cc][n++];
      }
    for (int k = 0; k < K; k++) {
      A[k][k] += ridge;
      g[k] = ld * tot[cc][NA + k];
    }
    for (int k = 0; k < K; k++) {
      P.sc->g[cc * K + k] = g[k];
      for (int l = 0; l < K; l++) P.sc->A[(cc * K + k) * K + l] = A[k][l];
    }
    if (solve) {
      bool ok = true;
      for (int j = 0; j < K && ok; j++) {
        double s = A[j][j];
        for (int m = 0; m < j; m++) s -= L[j][m] * L[j][m];
        if (!(s > 0.0)) {
          ok = false;
          break;
        }
        L[j][j] = sqrt(s);
        for (int i = j + 1; i < K; i++) {
          double t = A[i][j];
          for (int m = 0; m < j; m++) t -= L[i][m] * L[j][m];
          L[i][j] = t / L[j][j];
        }
      }
      if (ok) {
        for (int i = 0; i < K; i++) {
          double t = g[i];
          for (int m = 0; m < i; m++) t -= L[i][m] * yv[m];
          yv[i] = t / L[i][i];
        }
        for (int i = K - 1; i >= 0; i--) {
          double t = yv[i];
          for (int m = i + 1; m < K; m++) t -= L[m][i] * xs[m];
          xs[i] = t / L[i][i];
        }
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

// Exact energy (eq:giv-energy), 8 FP64 sums into sc->energy.
template <int K>
__global__ void __launch_bounds__(NT) k_energy(Params P) {
  __shared__ ColorTable<K> ct;
  load_colors<K>(ct, P.col);
  const Weights& w = P.w;
  const int x = blockIdx.x * BX + threadIdx.x, y = blockIdx.y * BY + threadIdx.y;
  float E[8];
  for (int i = 0; i < 8; i++) E[i] = 0.f;
  if (x < P.W && y < P.H) {
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
    const double s = block_sum((double)E[i]);
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

}  // namespace gid
