// Chromaticity clustering of Sec. 4.1 on the GPU: the initial base colours and
// the per-pixel cluster labels the solve starts from.  See include/gid.h
// (gid_cluster) for the contract.
//
//   k_hist      chromaticity C = I / (I_R + I_G + I_B + 1e-6) per pixel, its bin
//               in a 10 x 10 x 10 histogram over [0, 1]^3 (shared-memory
//               atomics, then one global add per bin and block)
//   k_kmeans    one block: weighted k-means on the occupied bins (mid-points
//               weighted by population, at most k_max centres, initialised at
//               the most populated bins), then merging of centres closer than
//               the threshold (the smaller cluster joins the larger; population-
//               weighted centre), clusters ordered by population; FP64
//   k_assign    every pixel to its closest centre (FP64 distances of its FP32
//               chromaticity); per-block FP64 sums of RGB and counts
//   k_colors    one block: the block sums in a fixed order -> mean RGB per cluster
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "../../include/gid.h"
#include "gid_nvtx.h"

namespace gidcl {

constexpr int NB = 10, NBINS = NB * NB * NB, KMAX = GID_MAX_K, ITERS = 100;
constexpr int TPB = 256, ASSIGN_BLOCKS = 148 * 4;

__device__ __forceinline__ void chroma(const float* __restrict__ rgb, long HW, long i, float* C) {
  const float r = rgb[i], g = rgb[HW + i], b = rgb[2 * HW + i];
  const float s = (r + g) + b + 1e-6f;
  C[0] = r / s;
  C[1] = g / s;
  C[2] = b / s;
}

__device__ __forceinline__ int bin_of(const float* C) {
  int idx[3];
  for (int c = 0; c < 3; c++) {
    const int v = (int)(C[c] * (float)NB);
    idx[c] = v < NB - 1 ? (v > 0 ? v : 0) : NB - 1;
  }
  return (idx[0] * NB + idx[1]) * NB + idx[2];
}

__global__ void k_hist(const float* __restrict__ rgb, long HW, unsigned* __restrict__ hist) {
  __shared__ unsigned h[NBINS];
  for (int i = threadIdx.x; i < NBINS; i += blockDim.x) h[i] = 0u;
  __syncthreads();
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (long)gridDim.x * blockDim.x) {
    float C[3];
    chroma(rgb, HW, i, C);
    atomicAdd(&h[bin_of(C)], 1u);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < NBINS; i += blockDim.x)
    if (h[i]) atomicAdd(&hist[i], h[i]);
}

struct Clusters {
  int k;                  // clusters after merging
  double centre[KMAX][3];  // ordered by decreasing population
  double pop[KMAX];
};

// One block of NBINS (rounded up to 1024) threads: thread t owns bin t.
__global__ void __launch_bounds__(1024) k_kmeans(const unsigned* __restrict__ hist, int k_max, double merge_dist,
                                                 Clusters* __restrict__ out) {
  __shared__ double cen[KMAX][3];
  __shared__ double sum[KMAX][4];
  __shared__ int k_s, changed;
  __shared__ int assign[NBINS];
  const int t = threadIdx.x;
  const double w = t < NBINS ? (double)hist[t] : 0.0;
  const double x[3] = {((t / (NB * NB)) + 0.5) / NB, (((t / NB) % NB) + 0.5) / NB, ((t % NB) + 0.5) / NB};
  if (t < NBINS) assign[t] = -1;
  if (t == 0) {
    // initial centres: the k_max most populated bins (ties by bin index)
    int k = 0;
    bool taken[NBINS];
    for (int i = 0; i < NBINS; i++) taken[i] = false;
    for (; k < k_max; k++) {
      int best = -1;
      for (int i = 0; i < NBINS; i++)
        if (!taken[i] && hist[i] > 0u && (best < 0 || hist[i] > hist[best])) best = i;
      if (best < 0) break;
      taken[best] = true;
      cen[k][0] = ((best / (NB * NB)) + 0.5) / NB;
      cen[k][1] = (((best / NB) % NB) + 0.5) / NB;
      cen[k][2] = ((best % NB) + 0.5) / NB;
    }
    k_s = k;
  }
  __syncthreads();
  const int k = k_s;
  for (int it = 0; it < ITERS; it++) {
    if (t == 0) changed = 0;
    __syncthreads();
    if (t < NBINS && w > 0.0) {
      int bj = 0;
      double bd = 0.0;
      for (int j = 0; j < k; j++) {
        double d = 0.0;
        for (int c = 0; c < 3; c++) d += (x[c] - cen[j][c]) * (x[c] - cen[j][c]);
        if (j == 0 || d < bd) {
          bd = d;
          bj = j;
        }
      }
      if (bj != assign[t]) {
        assign[t] = bj;
        changed = 1;
      }
    }
    __syncthreads();
    if (!changed) break;
    if (t < k) {
      double s[4] = {0.0, 0.0, 0.0, 0.0};
      for (int i = 0; i < NBINS; i++)
        if (assign[i] == t) {
          const double wi = (double)hist[i];
          s[0] += wi * (((i / (NB * NB)) + 0.5) / NB);
          s[1] += wi * ((((i / NB) % NB) + 0.5) / NB);
          s[2] += wi * (((i % NB) + 0.5) / NB);
          s[3] += wi;
        }
      if (s[3] > 0.0)
        for (int c = 0; c < 3; c++) cen[t][c] = s[c] / s[3];
    }
    __syncthreads();
  }
  if (t < k) {
    double p = 0.0;
    for (int i = 0; i < NBINS; i++)
      if (assign[i] == t) p += (double)hist[i];
    sum[t][3] = p;
  }
  __syncthreads();
  if (t == 0) {
    // merging: closest pair below the threshold first; the smaller joins the larger
    bool alive[KMAX];
    double c2[KMAX][3], pw[KMAX];
    for (int j = 0; j < k; j++) {
      alive[j] = sum[j][3] > 0.0;
      pw[j] = sum[j][3];
      for (int c = 0; c < 3; c++) c2[j][c] = cen[j][c];
    }
    for (;;) {
      int ba = -1, bb = -1;
      double bd = 0.0;
      for (int a = 0; a < k; a++)
        for (int b = a + 1; b < k; b++) {
          if (!alive[a] || !alive[b]) continue;
          double d = 0.0;
          for (int c = 0; c < 3; c++) d += (c2[a][c] - c2[b][c]) * (c2[a][c] - c2[b][c]);
          d = sqrt(d);
          if (d < merge_dist && (ba < 0 || d < bd)) {
            bd = d;
            ba = a;
            bb = b;
          }
        }
      if (ba < 0) break;
      const int big = (pw[ba] >= pw[bb]) ? ba : bb, small = big == ba ? bb : ba;
      for (int c = 0; c < 3; c++) c2[big][c] = (pw[big] * c2[big][c] + pw[small] * c2[small][c]) / (pw[big] + pw[small]);
      pw[big] += pw[small];
      alive[small] = false;
    }
    // order by decreasing population (ties by index)
    int n = 0;
    bool used[KMAX];
    for (int j = 0; j < k; j++) used[j] = false;
    for (;;) {
      int best = -1;
      for (int j = 0; j < k; j++)
        if (alive[j] && !used[j] && (best < 0 || pw[j] > pw[best])) best = j;
      if (best < 0) break;
      used[best] = true;
      for (int c = 0; c < 3; c++) out->centre[n][c] = c2[best][c];
      out->pop[n] = pw[best];
      n++;
    }
    out->k = n;
  }
}

__global__ void k_assign(const float* __restrict__ rgb, long HW, const Clusters* __restrict__ cl,
                         uint8_t* __restrict__ labels, double* __restrict__ part) {
  __shared__ double s[KMAX][4];
  __shared__ double cen[KMAX][3];
  __shared__ int k;
  if (threadIdx.x == 0) k = cl->k;
  if (threadIdx.x < KMAX * 4) s[threadIdx.x / 4][threadIdx.x % 4] = 0.0;
  if (threadIdx.x < KMAX * 3) cen[threadIdx.x / 3][threadIdx.x % 3] = cl->centre[threadIdx.x / 3][threadIdx.x % 3];
  __syncthreads();
  double acc[KMAX][4];
  for (int j = 0; j < KMAX; j++)
    for (int c = 0; c < 4; c++) acc[j][c] = 0.0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < HW; i += (long)gridDim.x * blockDim.x) {
    float C[3];
    chroma(rgb, HW, i, C);
    int bj = 0;
    double bd = 0.0;
    for (int j = 0; j < k; j++) {
      double d = 0.0;
      for (int c = 0; c < 3; c++) d += ((double)C[c] - cen[j][c]) * ((double)C[c] - cen[j][c]);
      if (j == 0 || d < bd) {
        bd = d;
        bj = j;
      }
    }
    labels[i] = (uint8_t)bj;
    for (int j = 0; j < KMAX; j++)
      if (j == bj) {
        acc[j][0] += (double)rgb[i];
        acc[j][1] += (double)rgb[HW + i];
        acc[j][2] += (double)rgb[2 * HW + i];
        acc[j][3] += 1.0;
      }
  }
  // block sums: thread order within a warp, then warps in order (fixed)
  for (int j = 0; j < k; j++)
    for (int c = 0; c < 4; c++) {
      double v = acc[j][c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      acc[j][c] = v;
    }
  __shared__ double ws[TPB / 32][KMAX][4];
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < k; j++)
      for (int c = 0; c < 4; c++) ws[threadIdx.x >> 5][j][c] = acc[j][c];
  __syncthreads();
  if (threadIdx.x < KMAX * 4) {
    const int j = threadIdx.x / 4, c = threadIdx.x % 4;
    double v = 0.0;
    if (j < k)
      for (int q = 0; q < TPB / 32; q++) v += ws[q][j][c];
    part[(long)blockIdx.x * KMAX * 4 + threadIdx.x] = v;
  }
}

__global__ void k_colors(const double* __restrict__ part, int nblocks, const Clusters* __restrict__ cl,
                         float* __restrict__ b) {
  const int t = threadIdx.x;  // one (cluster, channel) per thread
  if (t >= KMAX * 3) return;
  const int j = t / 3, c = t % 3;
  if (j >= cl->k) return;
  double s = 0.0, n = 0.0;
  for (int q = 0; q < nblocks; q++) {
    s += part[(long)q * KMAX * 4 + j * 4 + c];
    n += part[(long)q * KMAX * 4 + j * 4 + 3];
  }
  b[j * 3 + c] = n > 0.0 ? (float)(s / n) : (float)cl->centre[j][c];
}

}  // namespace gidcl

using namespace gidcl;

static int cl_fail(char* errbuf, int errbuf_len, int code, const std::string& m) {
  if (errbuf && errbuf_len > 0) {
    std::strncpy(errbuf, m.c_str(), (size_t)errbuf_len - 1);
    errbuf[errbuf_len - 1] = '\0';
  }
  return code;
}

extern "C" int gid_cluster(int H, int W, const float* rgb_dev, int k_max, float merge_dist, void* stream,
                           uint8_t* labels_dev, float* b_host, int* k_out, char* errbuf, int errbuf_len) {
  gid::NvtxRange nvtx_range("gid_cluster");
  if (!rgb_dev || !labels_dev || !b_host || !k_out)
    return cl_fail(errbuf, errbuf_len, GID_ERR_INVALID_ARG, "NULL argument");
  if (H < 1 || W < 1 || (long)H * W > (1L << 28)) return cl_fail(errbuf, errbuf_len, GID_ERR_INVALID_ARG, "bad H, W");
  if (k_max < 1 || k_max > GID_MAX_K) return cl_fail(errbuf, errbuf_len, GID_ERR_INVALID_ARG, "k_max in 1..10");
  if (!(merge_dist >= 0.f)) return cl_fail(errbuf, errbuf_len, GID_ERR_INVALID_ARG, "merge distance >= 0");
  cudaStream_t s = (cudaStream_t)stream;
  const long HW = (long)H * W;
  const int nblk = (int)std::min<long>(ASSIGN_BLOCKS, (HW + TPB - 1) / TPB);
  char* scratch = nullptr;
  const size_t hist_b = NBINS * sizeof(unsigned), cl_b = (sizeof(Clusters) + 255) / 256 * 256,
               part_b = (size_t)nblk * KMAX * 4 * sizeof(double), b_b = KMAX * 3 * sizeof(float);
  cudaError_t e = cudaMalloc(&scratch, 256 + hist_b + cl_b + part_b + b_b);
  if (e != cudaSuccess) return cl_fail(errbuf, errbuf_len, GID_ERR_OOM, "cluster scratch");
  unsigned* hist = reinterpret_cast<unsigned*>(scratch);
  Clusters* cl = reinterpret_cast<Clusters*>(scratch + (hist_b + 255) / 256 * 256);
  double* part = reinterpret_cast<double*>(reinterpret_cast<char*>(cl) + cl_b);
  float* bdev = reinterpret_cast<float*>(reinterpret_cast<char*>(part) + part_b);
  e = cudaMemsetAsync(hist, 0, hist_b, s);
  if (e == cudaSuccess) {
    k_hist<<<nblk, TPB, 0, s>>>(rgb_dev, HW, hist);
    k_kmeans<<<1, 1024, 0, s>>>(hist, k_max, (double)merge_dist, cl);
    k_assign<<<nblk, TPB, 0, s>>>(rgb_dev, HW, cl, labels_dev, part);
    k_colors<<<1, KMAX * 3, 0, s>>>(part, nblk, cl, bdev);
    e = cudaGetLastError();
  }
  int k = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&k, &cl->k, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(b_host, bdev, b_b, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(scratch);
  if (e != cudaSuccess) return cl_fail(errbuf, errbuf_len, GID_ERR_CUDA, cudaGetErrorString(e));
  *k_out = k;
  return GID_OK;
}
