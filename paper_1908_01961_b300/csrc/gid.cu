// C ABI of the illumination decomposition solver: context, buffers, launch
// sequence.  See include/gid.h for the contract of every entry point.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/gid.h"
#include "gid_kernels.cuh"
#include "gid_net_internal.h"
#include "gid_nvtx.h"

using namespace gid;

struct gid_ctx {
  int H = 0, W = 0, K = 0, V = 0, pitch = 0;
  long plane = 0;
  gid_weights w{};
  cudaStream_t stream = nullptr;
  char* pool = nullptr;
  size_t pool_bytes = 0;
  float *I = nullptr, *C = nullptr, *Cprev = nullptr, *rprev = nullptr, *wsr = nullptr, *ws = nullptr, *wt = nullptr,
        *wtsum = nullptr;
  uint8_t* lab = nullptr;
  float *X = nullptr, *d = nullptr, *z = nullptr, *pA = nullptr, *pB = nullptr, *q = nullptr,
        *Minv = nullptr, *coef = nullptr;
  DevColors* col = nullptr;
  DevScalars* sc = nullptr;
  double* partial = nullptr;
  double* pcg_part = nullptr;
  int nbmax = 0;
  // staging for the host-buffer entry point (allocated on first use)
  float* st_rgb = nullptr;
  uint8_t* st_lab = nullptr;
  float *st_R = nullptr, *st_T = nullptr;
  // double-buffered staging and a copy stream for the pipelined video entry point
  struct Pipe {
    cudaStream_t cs = nullptr;
    float *rgb[2] = {nullptr, nullptr}, *R[2] = {nullptr, nullptr}, *T[2] = {nullptr, nullptr},
          *b[2] = {nullptr, nullptr};
    uint8_t* lab[2] = {nullptr, nullptr};
    cudaEvent_t up[2] = {}, ingested[2] = {}, solved[2] = {}, down[2] = {};
  } pipe;
  bool has_colors = false, has_frame = false, initialised = false, temporal_active = false;
  int frames_solved = 0;
  long long launches = 0;  // kernels launched by this context
  int apply_th = 4;        // rows per operator tile (set by frame size at creation; gid_set_apply_tile / gid_autotune)
  int pcg_blocks = 0;      // > 0: run the PCG loop as one cooperative launch of this many blocks
  int upd_cap = 148 * 4;   // vector-step blocks resident at once (SMs x blocks per SM)
  int dense_cap = 148;     // base-colour-step blocks resident at once
  bool persistent = false; // persistent PCG kernel selected (gid_set_apply_tile(0) / gid_autotune)
  bool resident = false;   // resident PCG kernel selected (gid_set_apply_tile(-1) / gid_autotune)
  bool fused = false;      // one-kernel PCG step selected (gid_set_apply_tile(rows | GID_PCG_FUSED))
  bool l2_window = false;  // the PCG launches carry an L2 persistence window over the coefficients (gid_set_l2_window)
  cudaAccessPolicyWindow l2win{};
  float* fbuf = nullptr;   // its odd-step z and M^-1 q buffers (2 x V planes, allocated on first use)
  ResTile res{};           // its tile geometry; res_blocks = 0 if the frame does not fit on chip
  CUtensorMap res_map;     // its coefficient stream: box [1 plane][TH + 1 rows][4 TX + 8 columns]
  int res_blocks = 0, res_threads = 0;
  size_t res_smem = 0;
  bool res_planned = false;
  float* zx = nullptr;     // its border exchange planes (2 x V planes, allocated on first use)
  double* xval = nullptr;  // its all-reduce slots [RES_ROWS][RES_NV][RES_MAXB] and arrival counters
  int last_m_inner = 0;    // PCG steps of the latest Gauss-Newton step (gid_pcg_history)
  bool record_rho = false;  // copy each PCG step's rho into the history (gid_set_pcg_history)
  bool hist_valid = false;  // the latest Gauss-Newton step recorded its history
  int precond = 0;          // GID_PRECOND_JACOBI or GID_PRECOND_BLOCK (gid_set_preconditioner)
  float* blk = nullptr;     // block-Jacobi blocks in Schur form, block_planes(K) planes (allocated on first use)
  int blk_blocks = 0;       // grid of the block-Jacobi vector step
  // CUDA graphs of gid_run's launch sequence, replayed on a context-owned stream
  struct Graph {
    int n, m, refine, temporal, th, kernel;
    cudaGraphExec_t exec;
    long long kernels;
  };
  // TMA tensor maps of a staged PCG vector per (base pointer, tile rows):
  // boxes [3][rows + 6][136] (reflectance) and [K + 1][rows + 2][136] (layers)
  struct Maps {
    const float* base;
    int th;
    CUtensorMap r, t;
  };
  std::vector<Maps> maps;
  CUtensorMap lin_map;      // the state X for the linearisation: box [V][BY + 6][BX + 8]
  bool map_failed = false;  // a tensor map could not be encoded (the launch was skipped)
  bool use_graph = true;
  std::vector<Graph> graphs;
  cudaStream_t gs = nullptr;
  cudaEvent_t gev_in = nullptr, gev_out = nullptr;
  // optional per-kernel CUDA-event timing (gid_profile)
  bool prof = false;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_kind;  // kind of the kernel that ends at event i + 1
  double prof_ms[GID_NUM_KINDS] = {0};
  long long prof_n[GID_NUM_KINDS] = {0};
  std::string err;
};

static std::string g_create_err;

#define GID_TRY_CUDA(ctx, call)                                                             \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) return fail((ctx), GID_ERR_CUDA, #call, cudaGetErrorString(e_)); \
  } while (0)

static int fail(gid_ctx* ctx, int code, const char* what, const char* detail = nullptr) {
  std::string m = what;
  if (detail) m += std::string(": ") + detail;
  if (ctx)
    ctx->err = m;
  else
    g_create_err = m;
  return code;
}

// Wraps one kernel launch: counts it and, when profiling, brackets it with events.
template <class F>
static void launch(gid_ctx* c, int kind, F f) {
  const size_t i = c->ev_kind.size();
  if (c->prof && i + 1 < c->ev.size()) {
    // a chain of events: one before the first kernel, one after each kernel, so
    // that each kernel owns the time since the previous one ended (its launch
    // gap included) and the kernels partition the profiled time exactly
    if (i == 0) cudaEventRecord(c->ev[0], c->stream);
    f();
    cudaEventRecord(c->ev[i + 1], c->stream);
    c->ev_kind.push_back(kind);
  } else {
    f();
  }
  c->launches++;
}

static Weights to_dev(const gid_weights& w) {
  Weights d;
  d.ld = w.lambda_data;
  d.lcl = w.lambda_clustering;
  d.lrs = w.lambda_rsparsity;
  d.p = w.p;
  d.lrc = w.lambda_rconsistency;
  d.lm = w.lambda_monochrome;
  d.lis = w.lambda_isparsity;
  d.lsm = w.lambda_smoothness;
  d.lnn = w.lambda_nonneg;
  d.lIR = w.lambda_IR;
  d.lCR = w.lambda_CR;
  d.eps = w.eps;
  d.sharp = w.retinex_sharpness;
  d.tau = w.consistency_tau;
  d.nonneg_strict = w.nonneg_strict;
  d.irls_half = w.irls_half;
  d.rcluster_follows_b = w.rcluster_follows_b;
  return d;
}

static Params params(const gid_ctx* c) {
  Params P;
  memset(&P, 0, sizeof(P));
  P.H = c->H;
  P.W = c->W;
  P.pitch = c->pitch;
  P.plane = c->plane;
  P.w = to_dev(c->w);
  P.I = c->I;
  P.lab = c->lab;
  P.wsr = c->wsr;
  P.ws = c->ws;
  P.wt = c->wt;
  P.wtsum = c->wtsum;
  P.rprev = c->rprev;
  P.ns = c->w.n_spatial_pairs;
  P.nt = c->w.n_temporal_pairs;
  P.temporal = c->temporal_active ? 1 : 0;
  for (int i = 0; i < 2 * GID_MAX_PAIRS; i++) {
    P.off_s[i] = c->w.spatial_offsets[i];
    P.off_t[i] = c->w.temporal_offsets[i];
  }
  P.X = c->X;
  P.d = c->d;
  P.z = c->z;
  P.q = c->q;
  P.Minv = c->Minv;
  P.coef = c->coef;
  P.blk = c->blk;
  P.col = c->col;
  P.sc = c->sc;
  P.partial = c->partial;
  P.pcg_part = c->pcg_part;
  P.nbmax = c->nbmax;
  P.zx = c->zx;
  P.xval = c->xval;
  return P;
}

// How the PCG loop of a Gauss-Newton step runs: 0 one operator and one vector
// kernel per step, 1 the persistent cooperative kernel, 2 the resident one.
static void l2_release(gid_ctx* c);

// 0: operator and vector kernel per PCG step; 1: persistent; 2: resident; 3: fused step
static int pcg_kernel(const gid_ctx* c) {
  if (c->resident && c->res_blocks > 0) return 2;
  if (c->persistent && c->pcg_blocks > 0) return 1;
  if (c->fused && c->fbuf) return 3;
  return 0;
}

static dim3 pix_grid(const gid_ctx* c) { return dim3((c->W + BX - 1) / BX, (c->H + BY - 1) / BY); }
// Blocks per colour channel of the base-colour step: the three channels
// together fill one wave of resident blocks, each streaming its share of the
// pitched planes as float4.
static int dense_blocks(const gid_ctx* c) {
  return (int)std::max(1L, std::min((c->plane / 4 + 255) / 256, (long)std::max(1, c->dense_cap / 3)));
}
// Blocks of the PCG operator step for the context's tile shape.
static int apply_blocks(const gid_ctx* c) { return ((c->W + VTW - 1) / VTW) * ((c->H + c->apply_th - 1) / c->apply_th); }
// Blocks of the PCG vector step: exactly the blocks that are resident at once
// (one wave), striding over the planes; a partial second wave would run a
// quarter of the work on a fraction of the SMs.
static int update_blocks(const gid_ctx* c) {
  const long items = (long)c->V * (c->plane / 4);
  return (int)std::max(1L, std::min((items + 255) / 256, (long)c->upd_cap));
}
// Blocks of the PCG vector step that writes the <r, z> partials the next operator step reads.
static int vector_blocks(const gid_ctx* c) { return c->precond ? c->blk_blocks : update_blocks(c); }

// ---------------------------------------------------------------- TMA tensor maps

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 3-D tensor map of V pitched planes at `base` with the given box (x, y, planes).
static bool encode_planes(const gid_ctx* c, CUtensorMap* map, const float* base, cuuint32_t bx, cuuint32_t by,
                          cuuint32_t bz) {
  auto fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->H, (cuuint64_t)c->V};
  const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * sizeof(float), (cuuint64_t)c->plane * sizeof(float)};
  const cuuint32_t box[3] = {bx, by, bz};
  const cuuint32_t es[3] = {1u, 1u, 1u};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(base), dims, strides, box, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Tensor maps of the V planes at `base` (pitched like every context plane) for
// an operator tile of `th` rows; nullptr if the driver cannot encode them.
static const gid_ctx::Maps* tile_maps(gid_ctx* c, const float* base, int th) {
  for (const auto& m : c->maps)
    if (m.base == base && m.th == th) return &m;
  gid_ctx::Maps m;
  m.base = base;
  m.th = th;
  if (!encode_planes(c, &m.r, base, VRW, th + 2 * AHR, 3) || !encode_planes(c, &m.t, base, VRW, th + 2, c->K + 1))
    return nullptr;
  c->maps.push_back(m);
  return &c->maps.back();
}

// ---------------------------------------------------------------- K dispatch

// Operator tile rows of the work-list launches: 4 (four 128-thread blocks per
// SM, so one block's staging overlaps another's arithmetic).  Over the 24-video
// batch (many tiles, HBM-bound) 128 x 4 tiles ran at 46.3 Mpx/s, 128 x 8 at 45.7,
// 128 x 16 at 43.3 and 128 x 17 (the single 640 x 480 frame's one-wave tile) at
// 41.4.
constexpr int WL_TH = 4;

template <int K>
struct Launch {
  static void linearize(const gid_ctx* c, int mode, float* g, float* dg) {
    k_linearize<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c), mode, g, dg, c->lin_map);
  }
  // k_apply and k_update are launched as programmatic dependents of the kernel
  // before them: each may start (prefetch, colour table) while that kernel
  // drains, and waits on it in-kernel (griddepcontrol.wait) before reading
  // anything it wrote.  After any other kernel the launch is ordered as usual.
  template <class... KA, class... A>
  static void launch_pdl(const gid_ctx* c, void (*kern)(KA...), dim3 grid, dim3 block, size_t smem, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (c->l2_window) {
      attr[1].id = cudaLaunchAttributeAccessPolicyWindow;
      attr[1].val.accessPolicyWindow = c->l2win;
      cfg.numAttrs = 2;
    }
    cudaLaunchKernelEx(&cfg, kern, args...);
  }
  template <int TH>
  static void apply_th(const gid_ctx* c, int mode, int first, int it, const float* pin, float* pout, float* qout) {
    const size_t smem = sizeof(ApplyTile<K, TH>);
    const dim3 grid((c->W + VTW - 1) / VTW, (c->H + TH - 1) / TH);
    const gid_ctx::Maps* m = tile_maps(const_cast<gid_ctx*>(c), mode == 0 ? c->z : pin, TH);
    if (!m) {  // reported by the caller's launch check
      const_cast<gid_ctx*>(c)->map_failed = true;
      return;
    }
    launch_pdl(c, k_apply<K, TH>, grid, dim3(BX, TH), smem, params(c), mode, first, it, vector_blocks(c), pin, pout,
               qout, m->r, m->t);
  }
  // Fused PCG step `it` (k_pcg_step): z and M^-1 q alternate between the
  // context's buffers (z, q) for even steps and fbuf for odd ones.
  template <int TH>
  static void pcg_step_th(const gid_ctx* c, int it) {
    float* zb[2] = {c->z, c->fbuf};
    float* mb[2] = {c->q, c->fbuf + (long)c->V * c->plane};
    const float* zin = zb[(it - 1) & 1];
    const float* mqin = mb[(it - 1) & 1];
    const gid_ctx::Maps* m = tile_maps(const_cast<gid_ctx*>(c), zin, TH);
    const gid_ctx::Maps* mq = tile_maps(const_cast<gid_ctx*>(c), mqin, TH);
    if (!m || !mq) {
      const_cast<gid_ctx*>(c)->map_failed = true;
      return;
    }
    const dim3 grid((c->W + VTW - 1) / VTW, (c->H + TH - 1) / TH);
    launch_pdl(c, k_pcg_step<K, TH>, grid, dim3(BX, TH), fused_smem_bytes<K, TH>(), params(c), it, apply_blocks(c),
               zin, zb[it & 1], mqin, mb[it & 1], c->pA, m->r, m->t, mq->r, mq->t);
  }
  static void pcg_step(const gid_ctx* c, int it) {
    switch (c->apply_th) {
      case 2: pcg_step_th<2>(c, it); break;
      case 4: pcg_step_th<4>(c, it); break;
      case 17: pcg_step_th<17>(c, it); break;
      default: pcg_step_th<8>(c, it); break;
    }
  }
  // Opt every operator tile shape in to its dynamic shared memory (before any graph capture).
  static void prepare(const gid_ctx*) {
    cudaFuncSetAttribute(k_pcg_step<K, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem_bytes<K, 2>());
    cudaFuncSetAttribute(k_pcg_step<K, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem_bytes<K, 4>());
    cudaFuncSetAttribute(k_pcg_step<K, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem_bytes<K, 8>());
    cudaFuncSetAttribute(k_pcg_step<K, 17>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fused_smem_bytes<K, 17>());
    cudaFuncSetAttribute(k_apply<K, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, 2>));
    cudaFuncSetAttribute(k_apply<K, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, 4>));
    cudaFuncSetAttribute(k_apply<K, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, 8>));
    cudaFuncSetAttribute(k_apply<K, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, 16>));
    cudaFuncSetAttribute(k_apply<K, 17>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, 17>));
    cudaFuncSetAttribute(k_apply_multi<K, WL_TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)sizeof(ApplyTile<K, WL_TH>));
  }
  static void apply(const gid_ctx* c, int mode, int first, int it, const float* pin, float* pout, float* qout) {
    switch (c->apply_th) {
      case 2: apply_th<2>(c, mode, first, it, pin, pout, qout); break;
      case 4: apply_th<4>(c, mode, first, it, pin, pout, qout); break;
      case 16: apply_th<16>(c, mode, first, it, pin, pout, qout); break;
      case 17: apply_th<17>(c, mode, first, it, pin, pout, qout); break;
      default: apply_th<8>(c, mode, first, it, pin, pout, qout); break;
    }
  }
  // The persistent PCG loop: one block per SM of 17 x 32 threads; returns the launch error.
  static cudaError_t pcg(const gid_ctx* c, int m_inner, int last_mode) {
    constexpr int TH = 17;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->pcg_blocks);
    cfg.blockDim = dim3(BX, TH);
    cfg.dynamicSmemBytes = sizeof(ApplyTile<K, TH>);
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg<K, TH>, params(c), m_inner, last_mode, c->pA, c->q);
  }
  // Co-resident blocks of the persistent PCG kernel (0 if it cannot run here).
  static int pcg_capacity(const gid_ctx*) {
    constexpr int TH = 17;
    cudaFuncSetAttribute(k_pcg<K, TH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(ApplyTile<K, TH>));
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<K, TH>, BX * TH, sizeof(ApplyTile<K, TH>)) !=
        cudaSuccess)
      return 0;
    return coop ? sms * per_sm : 0;
  }
  // The resident PCG loop: one cooperative launch of res_blocks blocks.
  static cudaError_t resident(const gid_ctx* c, int m_inner, int last_mode) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->res_blocks);
    cfg.blockDim = dim3(c->res_threads);
    cfg.dynamicSmemBytes = c->res_smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_resident<K>, params(c), c->res, m_inner, last_mode, c->q, c->res_map);
  }
  // Tile geometry of the resident PCG kernel for this frame on this device:
  // among tiles of 4 TX x TH pixels (TX x TH <= RES_MAXT threads, shared
  // memory within the per-block limit) whose count fits the co-resident
  // blocks, the smallest tile (every phase waits for the slowest block) but
  // none below 512 pixels while fewer blocks can do (small frames: fewer
  // participants in every grid barrier), then the fewest blocks, then the
  // smallest staged halo.  res_blocks stays 0 if none fits.
  static void res_plan(gid_ctx* c) {
    c->res_planned = true;
    c->res_blocks = 0;
    int dev = 0, sms = 0, coop = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa;
    if (!coop || sms < 1 || cudaFuncGetAttributes(&fa, k_pcg_resident<K>) != cudaSuccess) return;
    const long limit = (long)optin - (long)fa.sharedSizeBytes;
    long best_area = -1, best_halo = 0, best_nb = 0;
    ResTile best{};
    for (int TX = 2; res_threads(TX, 1) <= RES_MAXT; TX++)
      for (int TH = 1; res_threads(TX, TH) <= RES_MAXT; TH++) {
        const long smem = res_smem_bytes(K, TX, TH);
        if (smem > limit) break;
        const long ntx = (c->W + 4 * TX - 1) / (4 * TX), nb = ntx * ((c->H + TH - 1) / TH);
        if (nb > sms) continue;
        const long area = std::max(4L * TX * TH, 512L), halo = (4L * TX + 8) * (TH + 6) - 4L * TX * TH;
        if (best_area < 0 || area < best_area || (area == best_area && nb < best_nb) ||
            (area == best_area && nb == best_nb && halo < best_halo)) {
          best_area = area;
          best_halo = halo;
          best_nb = nb;
          best = ResTile{TX, TH, (int)ntx, 4 * TX + 8};
        }
      }
    if (best_area < 0) return;
    const size_t smem = (size_t)res_smem_bytes(K, best.TX, best.TH);
    const int threads = res_threads(best.TX, best.TH);
    int per_sm = 0;
    if (cudaFuncSetAttribute(k_pcg_resident<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_resident<K>, threads, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      return;
    }
    const int nb = best.ntx * ((c->H + best.TH - 1) / best.TH);
    if (nb > sms * per_sm || nb > RES_MAXB) return;
    c->res = best;
    c->res_threads = threads;
    c->res_smem = smem;
    c->res_blocks = nb;
  }
  // The persistent work list of a batch group with this K: co-resident blocks
  // per SM (0 if it cannot run cooperatively), and its launch.
  static int pcg_multi_capacity() {
    int dev = 0, sms = 0, coop = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop ||
        cudaFuncSetAttribute(k_pcg_multi<K, WL_TH>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sizeof(ApplyTile<K, WL_TH>)) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_multi<K, WL_TH>, BX * WL_TH,
                                                      sizeof(ApplyTile<K, WL_TH>)) != cudaSuccess) {
      cudaGetLastError();
      return 0;
    }
    return sms * per_sm;
  }
  static cudaError_t pcg_multi(cudaStream_t s, const MultiVideo* vids, int nv, const CUtensorMap* maps, int tiles,
                               int upd, int m_inner, DevScalars* bar, int blocks) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(BX, WL_TH);
    cfg.dynamicSmemBytes = sizeof(ApplyTile<K, WL_TH>);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_pcg_multi<K, WL_TH>, vids, nv, maps, tiles, upd, m_inner, bar);
  }
  // Work-list PCG steps of a batch's videos with this K (operator tiles of 128 x WL_TH).
  static void apply_multi(cudaStream_t s, const MultiVideo* vids, int nv, const CUtensorMap* maps, int first, int it,
                          int blocks) {
    k_apply_multi<K, WL_TH><<<blocks, dim3(BX, WL_TH), sizeof(ApplyTile<K, WL_TH>), s>>>(vids, nv, maps, first, it);
  }
  static void update_multi(cudaStream_t s, const MultiVideo* vids, int nv, int it, int last, int blocks) {
    k_update_multi<K><<<blocks, 256, 0, s>>>(vids, nv, it, last);
  }
  // Resident blocks of the base-colour step on this device (SMs x blocks per SM).
  static int dense_capacity(const gid_ctx*) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense<K, true>, 256, 0) != cudaSuccess ||
        per_sm < 1 || sms < 1)
      return 148;
    return std::min(sms * per_sm, 148 * 8);
  }
  // Resident blocks of the vector step on this device (SMs x blocks per SM).
  static int update_capacity(const gid_ctx*) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<K>, 256, 0) != cudaSuccess || per_sm < 1 ||
        sms < 1)
      return 148 * 4;
    return std::min(sms * per_sm, 148 * 32);
  }
  static void update(const gid_ctx* c, int it, const float* p, int last) {
    launch_pdl(c, k_update<K>, dim3(update_blocks(c)), dim3(256), 0, params(c), it, apply_blocks(c), p, last);
  }
  // Block-Jacobi: the factorisation and PCG start, and the vector step.
  static void block_factor(const gid_ctx* c) {
    k_block_factor<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c));
  }
  static void update_block(const gid_ctx* c, int it, const float* p, int last) {
    launch_pdl(c, k_update_block<K>, dim3(c->blk_blocks), dim3(256), 0, params(c), it, apply_blocks(c), p, last);
  }
  // Resident blocks of the block-Jacobi vector step (SMs x blocks per SM).
  static int block_capacity(const gid_ctx*) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update_block<K>, 256, 0) != cudaSuccess ||
        per_sm < 1 || sms < 1)
      return 148 * 2;
    return sms * per_sm;
  }
  static void dense(const gid_ctx* c, int solve) {
    k_dense<K, true><<<dim3(dense_blocks(c), 3), 256, 0, c->stream>>>(params(c), solve);
  }
  static void energy(const gid_ctx* c, const uint8_t* mask = nullptr) {
    k_energy<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c), mask);
  }
  static void init_cold(const gid_ctx* c) { k_init_cold<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c)); }
  static void fit_direct(const gid_ctx* c) { k_fit_direct<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c)); }
  static void recombine(const gid_ctx* c, const EditTable& e, const uint8_t* mask, float* out) {
    k_recombine<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c), e, mask, out);
  }
  static void readout(const gid_ctx* c, float* R, float* T) {
    k_readout<K><<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(params(c), R, T);
  }
};

#define GID_DISPATCH(ctx, fn, ...)               \
  switch ((ctx)->K) {                            \
    case 1: Launch<1>::fn(__VA_ARGS__); break;   \
    case 2: Launch<2>::fn(__VA_ARGS__); break;   \
    case 3: Launch<3>::fn(__VA_ARGS__); break;   \
    case 4: Launch<4>::fn(__VA_ARGS__); break;   \
    case 5: Launch<5>::fn(__VA_ARGS__); break;   \
    case 6: Launch<6>::fn(__VA_ARGS__); break;   \
    case 7: Launch<7>::fn(__VA_ARGS__); break;   \
    case 8: Launch<8>::fn(__VA_ARGS__); break;   \
    case 9: Launch<9>::fn(__VA_ARGS__); break;   \
    case 10: Launch<10>::fn(__VA_ARGS__); break; \
    default: break;                              \
  }

static int check_launch(gid_ctx* c, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(c, GID_ERR_CUDA, what, cudaGetErrorString(e));
  if (c->map_failed) {
    c->map_failed = false;
    return fail(c, GID_ERR_CUDA, what, "TMA tensor map of the operator tile could not be encoded");
  }
  return GID_OK;
}

// Reads and clears the device status word; synchronises the stream.
static int sync_status(gid_ctx* c) {
  int st = 0;
  GID_TRY_CUDA(c, cudaMemcpyAsync(&st, &c->sc->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  if (st) {
    int zero = 0;
    GID_TRY_CUDA(c, cudaMemcpyAsync(&c->sc->status, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
    GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    if (st & ST_BAD_LABEL) return fail(c, GID_ERR_INVALID_ARG, "a label was >= K (treated as 0)");
    if (st & ST_SINGULAR) return fail(c, GID_ERR_NUMERIC, "base-colour normal equations not positive definite");
    if (st & ST_TIMEOUT) return fail(c, GID_ERR_TIMEOUT, "a grid barrier of the persistent PCG kernel gave up waiting");
  }
  return GID_OK;
}

// ---------------------------------------------------------------- ABI

extern "C" void gid_default_weights(gid_weights* w) {
  if (!w) return;
  memset(w, 0, sizeof(*w));
  w->lambda_data = 5000.f;
  w->lambda_clustering = 200.f;
  w->lambda_rsparsity = 20.f;
  w->p = 1.f;
  w->lambda_rconsistency = 10.f;
  w->lambda_monochrome = 10.f;
  w->lambda_isparsity = 3.f;
  w->lambda_smoothness = 3.f;
  w->lambda_nonneg = 1000.f;
  w->lambda_IR = 10.f;
  w->lambda_CR = 100.f;
  w->eps = 0.002f;
  w->retinex_sharpness = 50.f;
  w->consistency_tau = 0.05f;
  w->nonneg_strict = 1;
  w->irls_half = 0;
  w->rcluster_follows_b = 0;
  w->temporal = 0;
  w->refine_base_colors = 1;
}

static bool weights_ok(const gid_weights* w) {
  if (w->n_spatial_pairs < 0 || w->n_spatial_pairs > GID_MAX_PAIRS) return false;
  if (w->n_temporal_pairs < 0 || w->n_temporal_pairs > GID_MAX_PAIRS) return false;
  for (int i = 0; i < 2 * w->n_spatial_pairs; i++)
    if (std::abs(w->spatial_offsets[i]) > 3) return false;
  for (int i = 0; i < 2 * w->n_temporal_pairs; i++)
    if (std::abs(w->temporal_offsets[i]) > 3) return false;
  if (!(w->eps > 0.f) || !(w->consistency_tau > 0.f)) return false;
  if (w->refine_base_colors < 0 || w->refine_base_colors > 2) return false;
  return true;
}

extern "C" int gid_create(int H, int W, int K, const gid_weights* w, void* stream, gid_ctx** out) {
  if (!out) return fail(nullptr, GID_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (H < 1 || W < 1 || K < 1 || K > GID_MAX_K) return fail(nullptr, GID_ERR_INVALID_ARG, "bad H, W or K");
  if ((long)H * W > (1L << 28)) return fail(nullptr, GID_ERR_INVALID_ARG, "frame too large");
  gid_weights def;
  gid_default_weights(&def);
  if (!w) w = &def;
  if (!weights_ok(w)) return fail(nullptr, GID_ERR_INVALID_ARG, "bad weights (pairs, offsets, eps, tau or flags)");
  int dev_count = 0;
  cudaError_t e = cudaGetDeviceCount(&dev_count);
  if (e != cudaSuccess || dev_count < 1)
    return fail(nullptr, GID_ERR_CUDA, "no CUDA device", e != cudaSuccess ? cudaGetErrorString(e) : nullptr);
  gid_ctx* c = new (std::nothrow) gid_ctx();
  if (!c) return fail(nullptr, GID_ERR_OOM, "host allocation");
  c->H = H;
  c->W = W;
  c->K = K;
  c->V = K + 4;
  c->w = *w;
  c->stream = (cudaStream_t)stream;
  c->pitch = (W + 31) / 32 * 32;
  c->plane = (long)H * c->pitch;
  const int ns = std::max(1, w->n_spatial_pairs), nt = std::max(1, w->n_temporal_pairs);
  // planes: I 3, C 3, Cprev 3, rprev 3, wsr 1, ws ns, wt nt, wtsum 1, X d z pA pB q Minv 7V, coefficients
  const long nplanes = 3 + 3 + 3 + 3 + 1 + ns + nt + 1 + 7L * c->V + coef_planes(K, w->n_spatial_pairs);
  const size_t fbytes = (size_t)nplanes * c->plane * sizeof(float) + 256 * (size_t)nplanes;
  const size_t lbytes = ((size_t)c->plane + 255) / 256 * 256;
  // launch shapes that size the reduction buffers below
  switch (c->K) {
    case 1: c->upd_cap = Launch<1>::update_capacity(c); break;
    case 2: c->upd_cap = Launch<2>::update_capacity(c); break;
    case 3: c->upd_cap = Launch<3>::update_capacity(c); break;
    case 4: c->upd_cap = Launch<4>::update_capacity(c); break;
    case 5: c->upd_cap = Launch<5>::update_capacity(c); break;
    case 6: c->upd_cap = Launch<6>::update_capacity(c); break;
    case 7: c->upd_cap = Launch<7>::update_capacity(c); break;
    case 8: c->upd_cap = Launch<8>::update_capacity(c); break;
    case 9: c->upd_cap = Launch<9>::update_capacity(c); break;
    default: c->upd_cap = Launch<10>::update_capacity(c); break;
  }
  switch (c->K) {
    case 1: c->dense_cap = Launch<1>::dense_capacity(c); break;
    case 2: c->dense_cap = Launch<2>::dense_capacity(c); break;
    case 3: c->dense_cap = Launch<3>::dense_capacity(c); break;
    case 4: c->dense_cap = Launch<4>::dense_capacity(c); break;
    case 5: c->dense_cap = Launch<5>::dense_capacity(c); break;
    case 6: c->dense_cap = Launch<6>::dense_capacity(c); break;
    case 7: c->dense_cap = Launch<7>::dense_capacity(c); break;
    case 8: c->dense_cap = Launch<8>::dense_capacity(c); break;
    case 9: c->dense_cap = Launch<9>::dense_capacity(c); break;
    default: c->dense_cap = Launch<10>::dense_capacity(c); break;
  }
  cudaGetLastError();
  {
    // default operator tile (before any gid_autotune): 17 rows where the frame's
    // 128 x 17 tiles fit in one wave of one block per SM, else 4 rows (four
    // blocks per SM; many tiles, where small tiles overlap best)
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long n17 = (long)((W + VTW - 1) / VTW) * ((H + 16) / 17);
    c->apply_th = sms > 0 && n17 <= sms ? 17 : 4;
  }
  const long nb = std::max((long)pix_grid(c).x * pix_grid(c).y, (long)((W + VTW - 1) / VTW) * ((H + 1) / 2));
  const long nb_update = (c->plane / 4 + 255) / 256 * c->V;
  const long npart = std::max({nb * 8, nb_update, (long)dense_blocks(c) * 3 * (GID_MAX_K * (GID_MAX_K + 1) / 2 + GID_MAX_K)});
  const size_t pbytes = (size_t)npart * sizeof(double);
  c->nbmax = (int)std::max({(long)update_blocks(c), (long)((W + VTW - 1) / VTW) * ((H + 1) / 2), 148L * 32});
  const size_t ppbytes = sizeof(double) * 2 * PART_KINDS * (size_t)c->nbmax;
  c->pool_bytes = fbytes + lbytes + 256 * 9 + sizeof(DevColors) + sizeof(DevScalars) + pbytes + ppbytes;
  e = cudaMalloc(&c->pool, c->pool_bytes);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, GID_ERR_OOM, "cudaMalloc", cudaGetErrorString(e));
  }
  char* p = c->pool;
  auto take = [&](size_t bytes) {
    char* r = p;
    p += (bytes + 255) / 256 * 256;
    return r;
  };
  auto planes = [&](long n) { return (float*)take((size_t)n * c->plane * sizeof(float)); };
  c->I = planes(3);
  c->C = planes(3);
  c->Cprev = planes(3);
  c->rprev = planes(3);
  c->wsr = planes(1);
  c->ws = planes(ns);
  c->wt = planes(nt);
  c->wtsum = planes(1);
  // z, p, q and the coefficients last and contiguous: the PCG loop re-reads them
  // every step, and one L2 window (gid_set_l2_window) covers the coefficients and
  // as many of q, p, z as fit (at 640 x 480 K = 6: p and q; p and q in the window
  // measured 35.4 us per PCG step, z and q 35.8, the coefficients alone 37.4)
  c->X = planes(c->V);
  c->d = planes(c->V);
  c->pB = planes(c->V);
  c->Minv = planes(c->V);
  c->z = planes(c->V);
  c->pA = planes(c->V);
  c->q = planes(c->V);
  c->coef = planes(coef_planes(K, w->n_spatial_pairs));
  c->lab = (uint8_t*)take(lbytes);
  c->col = (DevColors*)take(sizeof(DevColors));
  c->sc = (DevScalars*)take(sizeof(DevScalars));
  c->partial = (double*)take(pbytes);
  c->pcg_part = (double*)take(ppbytes);
  if ((size_t)(p - c->pool) > c->pool_bytes) {
    cudaFree(c->pool);
    delete c;
    return fail(nullptr, GID_ERR_OOM, "internal pool layout");
  }
  GID_DISPATCH(c, prepare, c);
  if (!tile_maps(c, c->z, c->apply_th) || !encode_planes(c, &c->lin_map, c->X, LIN_C, LIN_R, c->V)) {
    cudaFree(c->pool);
    delete c;
    return fail(nullptr, GID_ERR_CUDA, "cuTensorMapEncodeTiled unavailable or failed for the operator tile");
  }
  switch (c->K) {
    case 1: c->pcg_blocks = Launch<1>::pcg_capacity(c); break;
    case 2: c->pcg_blocks = Launch<2>::pcg_capacity(c); break;
    case 3: c->pcg_blocks = Launch<3>::pcg_capacity(c); break;
    case 4: c->pcg_blocks = Launch<4>::pcg_capacity(c); break;
    case 5: c->pcg_blocks = Launch<5>::pcg_capacity(c); break;
    case 6: c->pcg_blocks = Launch<6>::pcg_capacity(c); break;
    case 7: c->pcg_blocks = Launch<7>::pcg_capacity(c); break;
    case 8: c->pcg_blocks = Launch<8>::pcg_capacity(c); break;
    case 9: c->pcg_blocks = Launch<9>::pcg_capacity(c); break;
    default: c->pcg_blocks = Launch<10>::pcg_capacity(c); break;
  }
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemsetAsync(c->pool, 0, c->pool_bytes, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    cudaFree(c->pool);
    delete c;
    return fail(nullptr, GID_ERR_CUDA, "cudaMemset", cudaGetErrorString(e));
  }
  *out = c;
  return GID_OK;
}

extern "C" void gid_destroy(gid_ctx* c) {
  if (!c) return;
  if (c->stream)
    cudaStreamSynchronize(c->stream);
  else
    cudaDeviceSynchronize();
  for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  if (c->gs) {
    cudaStreamSynchronize(c->gs);
    cudaStreamDestroy(c->gs);
    cudaEventDestroy(c->gev_in);
    cudaEventDestroy(c->gev_out);
  }
  cudaFree(c->pool);
  cudaFree(c->blk);
  cudaFree(c->zx);
  cudaFree(c->fbuf);
  l2_release(c);
  cudaFree(c->xval);
  cudaFree(c->st_rgb);
  cudaFree(c->st_lab);
  cudaFree(c->st_R);
  cudaFree(c->st_T);
  if (c->pipe.cs) {
    cudaStreamSynchronize(c->pipe.cs);
    cudaStreamDestroy(c->pipe.cs);
    for (int i = 0; i < 2; i++) {
      cudaFree(c->pipe.rgb[i]);
      cudaFree(c->pipe.lab[i]);
      cudaFree(c->pipe.R[i]);
      cudaFree(c->pipe.T[i]);
      cudaFree(c->pipe.b[i]);
      cudaEventDestroy(c->pipe.up[i]);
      cudaEventDestroy(c->pipe.ingested[i]);
      cudaEventDestroy(c->pipe.solved[i]);
      cudaEventDestroy(c->pipe.down[i]);
    }
  }
  delete c;
}

extern "C" const char* gid_last_error(const gid_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

extern "C" int gid_set_base_colors(gid_ctx* c, const float* b_host) {
  if (!c || !b_host) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  DevColors h;
  memset(&h, 0, sizeof(h));
  for (int i = 0; i < c->K * 3; i++) {
    if (!std::isfinite(b_host[i]) || !(b_host[i] > 0.f))
      return fail(c, GID_ERR_INVALID_ARG, "base colours must be finite and > 0");
    h.b[i] = h.binit[i] = b_host[i];
    h.bd[i] = b_host[i];
  }
  GID_TRY_CUDA(c, cudaMemcpyAsync(c->col, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  c->has_colors = true;
  return GID_OK;
}

extern "C" int gid_get_base_colors(gid_ctx* c, float* b_host) {
  if (!c || !b_host) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  DevColors h;
  GID_TRY_CUDA(c, cudaMemcpyAsync(&h, c->col, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  int rc = sync_status(c);
  for (int i = 0; i < c->K * 3; i++) b_host[i] = h.b[i];
  return rc;
}

extern "C" int gid_set_frame(gid_ctx* c, const float* rgb_dev, const uint8_t* labels_dev) {
  gid::NvtxRange nvtx_range("gid_set_frame");
  if (!c || !rgb_dev || !labels_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  const bool temporal = c->w.temporal && c->w.n_temporal_pairs > 0 && c->frames_solved > 0;
  if (temporal) {
    // The solved frame becomes the previous frame: its r and its chromaticity.
    GID_TRY_CUDA(c, cudaMemcpyAsync(c->rprev, c->X, sizeof(float) * 3 * c->plane, cudaMemcpyDeviceToDevice,
                                    c->stream));
    std::swap(c->C, c->Cprev);
  }
  c->temporal_active = temporal;
  Params P = params(c);
  launch(c, GID_KIND_FRAME, [&] {
    k_ingest<<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(P, rgb_dev, labels_dev, c->K, c->C, c->lab, c->I);
  });
  if (int rc = check_launch(c, "k_ingest")) return rc;
  launch(c, GID_KIND_FRAME, [&] {
    k_prior_weights<<<pix_grid(c), dim3(BX, BY), 0, c->stream>>>(P, c->C, c->Cprev, c->wsr, c->ws, c->wt,
                                                                  c->wtsum);
  });
  if (int rc = check_launch(c, "k_prior_weights")) return rc;
  c->has_frame = true;
  return GID_OK;
}

extern "C" int gid_new_sequence(gid_ctx* c) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  launch(c, GID_KIND_INIT, [&] { k_reset_colors<<<1, 32, 0, c->stream>>>(c->col, 3 * c->K); });
  if (int rc = check_launch(c, "k_reset_colors")) return rc;
  c->frames_solved = 0;
  c->temporal_active = false;
  c->initialised = false;
  return GID_OK;
}

extern "C" int gid_init(gid_ctx* c, int mode) {
  gid::NvtxRange nvtx_range("gid_init");
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (!c->has_frame || !c->has_colors)
    return fail(c, GID_ERR_STATE, "gid_init needs gid_set_base_colors and gid_set_frame");
  if (mode == 0) {
    launch(c, GID_KIND_INIT, [&] { GID_DISPATCH(c, init_cold, c); });
    if (int rc = check_launch(c, "k_init_cold")) return rc;
  } else if (mode == 1) {
    if (!c->initialised) return fail(c, GID_ERR_STATE, "warm start needs a previous state");
  } else {
    return fail(c, GID_ERR_INVALID_ARG, "init mode must be 0 (cold) or 1 (warm)");
  }
  c->initialised = true;
  return GID_OK;
}

extern "C" int gid_base_color_step(gid_ctx* c) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (!c->has_frame || !c->initialised || !c->has_colors) return fail(c, GID_ERR_STATE, "no frame/state/colours");
  launch(c, GID_KIND_DENSE, [&] { GID_DISPATCH(c, dense, c, 1); });
  return check_launch(c, "k_dense");
}

extern "C" int gid_init_learned(gid_ctx* c, gid_net* net, float zero_below) {
  gid::NvtxRange nvtx_range("gid_init_learned");
  if (!c || !net) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (!(zero_below >= 0.f) || !std::isfinite(zero_below)) return fail(c, GID_ERR_INVALID_ARG, "zero_below >= 0");
  if (!c->has_frame || !c->has_colors)
    return fail(c, GID_ERR_STATE, "gid_init_learned needs gid_set_base_colors and gid_set_frame");
  if (gidnet_K(net) != c->K) return fail(c, GID_ERR_INVALID_ARG, "network and context have different K");
  if (c->H % 8 || c->W % 8) return fail(c, GID_ERR_INVALID_ARG, "learned start needs H and W multiples of 8");
  // the palette is the initial (clustered) base colours, index-aligned with b_1..b_K
  const float* palette = reinterpret_cast<const float*>(reinterpret_cast<const char*>(c->col) +
                                                        offsetof(DevColors, binit));
  std::string msg;
  // Indirect values below zero_below start at exactly zero: the sparse prior's
  // default state, which the reweighting of Sec. 5.3 keeps from overshooting
  // below zero (a strictly positive value has non-negativity weight zero).
  if (int rc = gidnet_infer_planes(net, c->H, c->W, c->I, c->plane, c->pitch, c->lab, palette, zero_below, c->X,
                                   c->stream, &c->launches, &msg))
    return fail(c, rc, "network forward", msg.c_str());
  // T_0 refit to the data term per pixel (closed form) on the predicted R and T_1..T_K
  launch(c, GID_KIND_INIT, [&] { GID_DISPATCH(c, fit_direct, c); });
  if (int rc = check_launch(c, "k_fit_direct")) return rc;
  if (c->w.refine_base_colors != 0) {
    launch(c, GID_KIND_DENSE, [&] { GID_DISPATCH(c, dense, c, 1); });
    if (int rc = check_launch(c, "k_dense")) return rc;
  }
  c->initialised = true;
  return GID_OK;
}

// With recording on: rho of PCG step m (published in rho2 by the operator step
// m, or by the PCG start for m = 1) into the history; an 8-byte device copy
// in the stream, so the kernels themselves carry nothing for it.
static void record_rho(gid_ctx* c, int m) {
  if (c->record_rho && m >= 2 && m - 1 < PCG_HIST)
    cudaMemcpyAsync(&c->sc->rho_hist[m - 1], &c->sc->rho2[m & 1], sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
}

static int enqueue_gn_step(gid_ctx* c, int m_inner, int last_mode) {
  c->last_m_inner = m_inner;
  c->hist_valid = c->record_rho || (pcg_kernel(c) != 0 && c->precond == GID_PRECOND_JACOBI);  // in-kernel history
  if (c->precond == GID_PRECOND_BLOCK) {
    launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, linearize, c, 3, (float*)nullptr, (float*)nullptr); });
    launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, block_factor, c); });
    if (int rc = check_launch(c, "k_linearize / k_block_factor")) return rc;
    for (int m = 1; m <= m_inner; m++) {
      launch(c, GID_KIND_APPLY,
             [&] { GID_DISPATCH(c, apply, c, 0, m == 1 ? 1 : 0, m, (const float*)c->pA, c->pA, c->q); });
      record_rho(c, m);
      launch(c, GID_KIND_UPDATE,
             [&] { GID_DISPATCH(c, update_block, c, m, (const float*)c->pA, m == m_inner ? last_mode : 0); });
    }
    return check_launch(c, "pcg (block-Jacobi)");
  }
  launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, linearize, c, 0, (float*)nullptr, (float*)nullptr); });
  if (int rc = check_launch(c, "k_linearize")) return rc;
  if (pcg_kernel(c) == 3) {
    // one fused kernel per PCG step, then the last step's vector update
    for (int m = 1; m <= m_inner; m++) launch(c, GID_KIND_APPLY, [&] { GID_DISPATCH(c, pcg_step, c, m); });
    launch(c, GID_KIND_UPDATE, [&] { GID_DISPATCH(c, update, c, m_inner, (const float*)c->pA, last_mode); });
    return check_launch(c, "k_pcg_step");
  }
  if (pcg_kernel(c) == 2) {
    cudaError_t e = cudaSuccess;
    launch(c, GID_KIND_PCG, [&] {
      switch (c->K) {
        case 1: e = Launch<1>::resident(c, m_inner, last_mode); break;
        case 2: e = Launch<2>::resident(c, m_inner, last_mode); break;
        case 3: e = Launch<3>::resident(c, m_inner, last_mode); break;
        case 4: e = Launch<4>::resident(c, m_inner, last_mode); break;
        case 5: e = Launch<5>::resident(c, m_inner, last_mode); break;
        case 6: e = Launch<6>::resident(c, m_inner, last_mode); break;
        case 7: e = Launch<7>::resident(c, m_inner, last_mode); break;
        case 8: e = Launch<8>::resident(c, m_inner, last_mode); break;
        case 9: e = Launch<9>::resident(c, m_inner, last_mode); break;
        default: e = Launch<10>::resident(c, m_inner, last_mode); break;
      }
    });
    if (e != cudaSuccess) return fail(c, GID_ERR_CUDA, "k_pcg_resident (cooperative launch)", cudaGetErrorString(e));
    return check_launch(c, "k_pcg_resident");
  }
  if (pcg_kernel(c) == 1) {
    cudaError_t e = cudaSuccess;
    launch(c, GID_KIND_PCG, [&] {
      switch (c->K) {
        case 1: e = Launch<1>::pcg(c, m_inner, last_mode); break;
        case 2: e = Launch<2>::pcg(c, m_inner, last_mode); break;
        case 3: e = Launch<3>::pcg(c, m_inner, last_mode); break;
        case 4: e = Launch<4>::pcg(c, m_inner, last_mode); break;
        case 5: e = Launch<5>::pcg(c, m_inner, last_mode); break;
        case 6: e = Launch<6>::pcg(c, m_inner, last_mode); break;
        case 7: e = Launch<7>::pcg(c, m_inner, last_mode); break;
        case 8: e = Launch<8>::pcg(c, m_inner, last_mode); break;
        case 9: e = Launch<9>::pcg(c, m_inner, last_mode); break;
        default: e = Launch<10>::pcg(c, m_inner, last_mode); break;
      }
    });
    if (e != cudaSuccess) return fail(c, GID_ERR_CUDA, "k_pcg (cooperative launch)", cudaGetErrorString(e));
    return check_launch(c, "k_pcg");
  }
  // p and q are updated in place (see k_apply); step m's scalars use partial slots m % 2
  for (int m = 1; m <= m_inner; m++) {
    launch(c, GID_KIND_APPLY,
           [&] { GID_DISPATCH(c, apply, c, 0, m == 1 ? 1 : 0, m, (const float*)c->pA, c->pA, c->q); });
    record_rho(c, m);
    launch(c, GID_KIND_UPDATE, [&] { GID_DISPATCH(c, update, c, m, (const float*)c->pA, m == m_inner ? last_mode : 0); });
  }
  return check_launch(c, "pcg");
}

static int enqueue_run(gid_ctx* c, int n_outer, int m_inner, bool refine) {
  for (int n = 0; n < n_outer; n++) {
    if (int rc = enqueue_gn_step(c, m_inner, 1)) return rc;
    if (refine) {
      launch(c, GID_KIND_DENSE, [&] { GID_DISPATCH(c, dense, c, 1); });
      if (int rc = check_launch(c, "k_dense")) return rc;
    }
  }
  return GID_OK;
}

// Capture the run's launch sequence once per (N, M, refinement, temporal pairs,
// tile shape) into a CUDA graph on the context's own stream; replay it fenced
// by events against the caller's stream (which may be the legacy default
// stream, where capture is not allowed).
static int run_graph(gid_ctx* c, int n_outer, int m_inner, bool refine) {
  if (!c->gs) {
    GID_TRY_CUDA(c, cudaStreamCreateWithFlags(&c->gs, cudaStreamNonBlocking));
    GID_TRY_CUDA(c, cudaEventCreateWithFlags(&c->gev_in, cudaEventDisableTiming));
    GID_TRY_CUDA(c, cudaEventCreateWithFlags(&c->gev_out, cudaEventDisableTiming));
  }
  const int temporal = c->temporal_active ? 1 : 0;
  gid_ctx::Graph* g = nullptr;
  for (auto& e : c->graphs)
    if (e.n == n_outer && e.m == m_inner && e.refine == (int)refine && e.temporal == temporal && e.th == c->apply_th &&
        e.kernel == pcg_kernel(c))
      g = &e;
  if (!g) {
    cudaStream_t user = c->stream;
    const long long l0 = c->launches;
    GID_TRY_CUDA(c, cudaStreamBeginCapture(c->gs, cudaStreamCaptureModeThreadLocal));
    c->stream = c->gs;
    int rc = enqueue_run(c, n_outer, m_inner, refine);
    c->stream = user;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(c->gs, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      c->launches = l0;
      return rc;
    }
    if (e != cudaSuccess) return fail(c, GID_ERR_CUDA, "cudaStreamEndCapture", cudaGetErrorString(e));
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(c, GID_ERR_CUDA, "cudaGraphInstantiate", cudaGetErrorString(e));
    c->graphs.push_back({n_outer, m_inner, (int)refine, temporal, c->apply_th, pcg_kernel(c), exec, c->launches - l0});
    c->launches = l0;
    g = &c->graphs.back();
  }
  GID_TRY_CUDA(c, cudaEventRecord(c->gev_in, c->stream));
  GID_TRY_CUDA(c, cudaStreamWaitEvent(c->gs, c->gev_in, 0));
  GID_TRY_CUDA(c, cudaGraphLaunch(g->exec, c->gs));
  GID_TRY_CUDA(c, cudaEventRecord(c->gev_out, c->gs));
  GID_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, c->gev_out, 0));
  c->launches += g->kernels;
  return GID_OK;
}

extern "C" int gid_run(gid_ctx* c, int n_outer, int m_inner) {
  gid::NvtxRange nvtx_range("gid_run");
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (n_outer < 0 || m_inner < 1) return fail(c, GID_ERR_INVALID_ARG, "n_outer >= 0 and m_inner >= 1");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "gid_run before gid_set_frame / gid_init");
  const bool refine = c->w.refine_base_colors == 1 || (c->w.refine_base_colors == 2 && c->frames_solved == 0);
  int rc = (c->use_graph && !c->prof && n_outer > 0) ? run_graph(c, n_outer, m_inner, refine)
                                                      : enqueue_run(c, n_outer, m_inner, refine);
  if (rc) return rc;
  c->frames_solved++;
  return GID_OK;
}

extern "C" int gid_set_graphs(gid_ctx* c, int enable) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  c->use_graph = enable != 0;
  return GID_OK;
}

extern "C" int gid_get_layers(gid_ctx* c, float* R_dev, float* T_dev) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (!c->initialised) return fail(c, GID_ERR_STATE, "no state");
  if (!R_dev && !T_dev) return GID_OK;
  launch(c, GID_KIND_READOUT, [&] { GID_DISPATCH(c, readout, c, R_dev, T_dev); });
  return check_launch(c, "k_readout");
}

extern "C" int gid_recombine(gid_ctx* c, const float* b_new_host, const float* gain_host, const uint8_t* mask_dev,
                             float* out_dev) {
  if (!c || !out_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (!c->initialised || !c->has_colors) return fail(c, GID_ERR_STATE, "no state / base colours");
  EditTable e;
  if (b_new_host) {
    for (int i = 0; i < 3 * c->K; i++) {
      if (!std::isfinite(b_new_host[i])) return fail(c, GID_ERR_INVALID_ARG, "new base colours must be finite");
      e.bn[i] = b_new_host[i];
    }
  } else {
    DevColors h;
    GID_TRY_CUDA(c, cudaMemcpyAsync(&h, c->col, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
    GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int i = 0; i < 3 * c->K; i++) e.bn[i] = h.b[i];
  }
  for (int k = 0; k < c->K; k++) {
    const float g = gain_host ? gain_host[k] : 1.f;
    if (!std::isfinite(g)) return fail(c, GID_ERR_INVALID_ARG, "layer gains must be finite");
    e.gain[k] = g;
  }
  launch(c, GID_KIND_READOUT, [&] { GID_DISPATCH(c, recombine, c, e, mask_dev, out_dev); });
  return check_launch(c, "k_recombine");
}

extern "C" int gid_get_state(gid_ctx* c, float* X_dev) {
  if (!c || !X_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  GID_TRY_CUDA(c, cudaMemcpy2DAsync(X_dev, sizeof(float) * c->W, c->X, sizeof(float) * c->pitch, sizeof(float) * c->W,
                                    (size_t)c->V * c->H, cudaMemcpyDeviceToDevice, c->stream));
  return GID_OK;
}

extern "C" int gid_set_state(gid_ctx* c, const float* X_dev) {
  if (!c || !X_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  GID_TRY_CUDA(c, cudaMemcpy2DAsync(c->X, sizeof(float) * c->pitch, X_dev, sizeof(float) * c->W, sizeof(float) * c->W,
                                    (size_t)c->V * c->H, cudaMemcpyDeviceToDevice, c->stream));
  if (c->pitch > c->W)  // padding columns are zero (a failed earlier solve may have left NaN there)
    GID_TRY_CUDA(c, cudaMemset2DAsync(c->X + c->W, sizeof(float) * c->pitch, 0, sizeof(float) * (c->pitch - c->W),
                                      (size_t)c->V * c->H, c->stream));
  c->initialised = true;
  return GID_OK;
}

extern "C" int gid_energy_region(gid_ctx* c, const uint8_t* mask_dev, double* total, double* per_term) {
  gid::NvtxRange nvtx_range("gid_energy");
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "no frame/state");
  launch(c, GID_KIND_ENERGY, [&] { GID_DISPATCH(c, energy, c, mask_dev); });
  if (int rc = check_launch(c, "k_energy")) return rc;
  double E[8];
  GID_TRY_CUDA(c, cudaMemcpyAsync(E, c->sc->energy, sizeof(E), cudaMemcpyDeviceToHost, c->stream));
  int rc = sync_status(c);
  double t = 0;
  for (int i = 0; i < 8; i++) t += E[i];
  if (per_term) memcpy(per_term, E, sizeof(E));
  if (total) *total = t;
  if (rc) return rc;
  if (!std::isfinite(t)) return fail(c, GID_ERR_NUMERIC, "energy is not finite");
  return GID_OK;
}

extern "C" int gid_energy(gid_ctx* c, double* total, double* per_term) {
  return gid_energy_region(c, nullptr, total, per_term);
}

extern "C" int gid_solve_frame_host(gid_ctx* c, const float* rgb_host, const uint8_t* labels_host, int init_mode,
                                    int n_outer, int m_inner, float* R_host, float* T_host, float* b_host) {
  gid::NvtxRange nvtx_range("gid_solve_frame_host");
  if (!c || !rgb_host || !labels_host) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  const size_t HW = (size_t)c->H * c->W;
  if (!c->st_rgb) {
    GID_TRY_CUDA(c, cudaMalloc(&c->st_rgb, 3 * HW * sizeof(float)));
    GID_TRY_CUDA(c, cudaMalloc(&c->st_lab, HW));
    GID_TRY_CUDA(c, cudaMalloc(&c->st_R, 3 * HW * sizeof(float)));
    GID_TRY_CUDA(c, cudaMalloc(&c->st_T, (size_t)(c->K + 1) * HW * sizeof(float)));
  }
  GID_TRY_CUDA(c, cudaMemcpyAsync(c->st_rgb, rgb_host, 3 * HW * sizeof(float), cudaMemcpyHostToDevice, c->stream));
  GID_TRY_CUDA(c, cudaMemcpyAsync(c->st_lab, labels_host, HW, cudaMemcpyHostToDevice, c->stream));
  if (int rc = gid_set_frame(c, c->st_rgb, c->st_lab)) return rc;
  if (int rc = gid_init(c, init_mode)) return rc;
  if (int rc = gid_run(c, n_outer, m_inner)) return rc;
  if (R_host || T_host) {
    if (int rc = gid_get_layers(c, c->st_R, c->st_T)) return rc;
    if (R_host)
      GID_TRY_CUDA(c, cudaMemcpyAsync(R_host, c->st_R, 3 * HW * sizeof(float), cudaMemcpyDeviceToHost, c->stream));
    if (T_host)
      GID_TRY_CUDA(c, cudaMemcpyAsync(T_host, c->st_T, (size_t)(c->K + 1) * HW * sizeof(float),
                                      cudaMemcpyDeviceToHost, c->stream));
  }
  if (b_host) return gid_get_base_colors(c, b_host);
  return sync_status(c);
}

extern "C" int gid_solve_video_host(gid_ctx* c, int n, const float* rgb_host, const uint8_t* labels_host,
                                    int first_init_mode, int n_outer, int m_inner, float* R_host, float* T_host,
                                    float* b_host) {
  gid::NvtxRange nvtx_range("gid_solve_video_host");
  if (!c || !rgb_host || !labels_host) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (n < 1) return fail(c, GID_ERR_INVALID_ARG, "n >= 1 frames");
  if (first_init_mode != 0 && first_init_mode != 1) return fail(c, GID_ERR_INVALID_ARG, "init mode 0 or 1");
  const size_t HW = (size_t)c->H * c->W, rgb_b = 3 * HW * sizeof(float), R_b = 3 * HW * sizeof(float),
               T_b = (size_t)(c->K + 1) * HW * sizeof(float), b_b = (size_t)c->K * 3 * sizeof(float);
  auto& pp = c->pipe;
  if (!pp.cs) {
    GID_TRY_CUDA(c, cudaStreamCreateWithFlags(&pp.cs, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++) {
      GID_TRY_CUDA(c, cudaMalloc(&pp.rgb[i], rgb_b));
      GID_TRY_CUDA(c, cudaMalloc(&pp.lab[i], HW));
      GID_TRY_CUDA(c, cudaMalloc(&pp.R[i], R_b));
      GID_TRY_CUDA(c, cudaMalloc(&pp.T[i], T_b));
      GID_TRY_CUDA(c, cudaMalloc(&pp.b[i], b_b));
      for (cudaEvent_t* e : {&pp.up[i], &pp.ingested[i], &pp.solved[i], &pp.down[i]})
        GID_TRY_CUDA(c, cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    }
  }
  // slot i's staging is reused every other frame: an upload waits for the
  // ingest of the frame two back, an output for the download of the frame two back
  auto upload = [&](int t) -> int {
    const int i = t & 1;
    if (t >= 2) GID_TRY_CUDA(c, cudaStreamWaitEvent(pp.cs, pp.ingested[i], 0));
    GID_TRY_CUDA(c, cudaMemcpyAsync(pp.rgb[i], rgb_host + (size_t)t * 3 * HW, rgb_b, cudaMemcpyHostToDevice, pp.cs));
    GID_TRY_CUDA(c, cudaMemcpyAsync(pp.lab[i], labels_host + (size_t)t * HW, HW, cudaMemcpyHostToDevice, pp.cs));
    GID_TRY_CUDA(c, cudaEventRecord(pp.up[i], pp.cs));
    return GID_OK;
  };
  if (int rc = upload(0)) return rc;
  const float* colors = reinterpret_cast<const float*>(reinterpret_cast<const char*>(c->col) + offsetof(DevColors, b));
  for (int t = 0; t < n; t++) {
    const int i = t & 1;
    GID_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, pp.up[i], 0));
    if (int rc = gid_set_frame(c, pp.rgb[i], pp.lab[i])) return rc;
    GID_TRY_CUDA(c, cudaEventRecord(pp.ingested[i], c->stream));
    if (t + 1 < n)
      if (int rc = upload(t + 1)) return rc;  // overlaps this frame's solve
    if (int rc = gid_init(c, t == 0 ? first_init_mode : 1)) return rc;
    if (int rc = gid_run(c, n_outer, m_inner)) return rc;
    if (t >= 2) GID_TRY_CUDA(c, cudaStreamWaitEvent(c->stream, pp.down[i], 0));
    if (R_host || T_host)
      if (int rc = gid_get_layers(c, pp.R[i], pp.T[i])) return rc;
    GID_TRY_CUDA(c, cudaMemcpyAsync(pp.b[i], colors, b_b, cudaMemcpyDeviceToDevice, c->stream));
    GID_TRY_CUDA(c, cudaEventRecord(pp.solved[i], c->stream));
    // download frame t on the copy stream while frame t + 1 is solved
    GID_TRY_CUDA(c, cudaStreamWaitEvent(pp.cs, pp.solved[i], 0));
    if (R_host) GID_TRY_CUDA(c, cudaMemcpyAsync(R_host + (size_t)t * 3 * HW, pp.R[i], R_b, cudaMemcpyDeviceToHost, pp.cs));
    if (T_host)
      GID_TRY_CUDA(c, cudaMemcpyAsync(T_host + (size_t)t * (c->K + 1) * HW, pp.T[i], T_b, cudaMemcpyDeviceToHost,
                                      pp.cs));
    if (b_host) GID_TRY_CUDA(c, cudaMemcpyAsync(b_host + (size_t)t * c->K * 3, pp.b[i], b_b, cudaMemcpyDeviceToHost, pp.cs));
    GID_TRY_CUDA(c, cudaEventRecord(pp.down[i], pp.cs));
  }
  GID_TRY_CUDA(c, cudaStreamSynchronize(pp.cs));
  return sync_status(c);
}

// ---------------------------------------------------------------- stages

extern "C" int gid_stage_precompute(gid_ctx* c, float* wsr_dev, float* omega_s_dev, float* omega_t_dev) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (!c->has_frame) return fail(c, GID_ERR_STATE, "no frame");
  auto out = [&](float* dst, const float* src, int n) -> int {
    if (!dst || n <= 0) return GID_OK;
    GID_TRY_CUDA(c, cudaMemcpy2DAsync(dst, sizeof(float) * c->W, src, sizeof(float) * c->pitch, sizeof(float) * c->W,
                                      (size_t)n * c->H, cudaMemcpyDeviceToDevice, c->stream));
    return GID_OK;
  };
  if (int rc = out(wsr_dev, c->wsr, 1)) return rc;
  if (int rc = out(omega_s_dev, c->ws, c->w.n_spatial_pairs)) return rc;
  if (omega_t_dev && c->w.n_temporal_pairs > 0) {
    if (c->temporal_active) return out(omega_t_dev, c->wt, c->w.n_temporal_pairs);
    GID_TRY_CUDA(c, cudaMemsetAsync(omega_t_dev, 0, sizeof(float) * c->w.n_temporal_pairs * c->H * c->W, c->stream));
  }
  return GID_OK;
}

// The stage calls reuse the PCG buffers (pA, pB, d) as scratch and copy into /
// out of the caller's contiguous arrays.
static int to_pitched(gid_ctx* c, float* dst, const float* src) {
  GID_TRY_CUDA(c, cudaMemcpy2DAsync(dst, sizeof(float) * c->pitch, src, sizeof(float) * c->W, sizeof(float) * c->W,
                                    (size_t)c->V * c->H, cudaMemcpyDeviceToDevice, c->stream));
  return GID_OK;
}
static int from_pitched(gid_ctx* c, float* dst, const float* src) {
  GID_TRY_CUDA(c, cudaMemcpy2DAsync(dst, sizeof(float) * c->W, src, sizeof(float) * c->pitch, sizeof(float) * c->W,
                                    (size_t)c->V * c->H, cudaMemcpyDeviceToDevice, c->stream));
  return GID_OK;
}

extern "C" int gid_stage_linearize(gid_ctx* c, float* g_dev, float* diag_dev) {
  if (!c || !g_dev || !diag_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "no frame/state");
  launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, linearize, c, 1, c->pA, c->pB); });
  if (int rc = check_launch(c, "k_linearize")) return rc;
  if (int rc = from_pitched(c, g_dev, c->pA)) return rc;
  return from_pitched(c, diag_dev, c->pB);
}

extern "C" int gid_stage_apply(gid_ctx* c, const float* p_dev, float* q_dev) {
  if (!c || !p_dev || !q_dev) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "no frame/state");
  if (int rc = to_pitched(c, c->pA, p_dev)) return rc;
  launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, linearize, c, 2, (float*)nullptr, (float*)nullptr); });
  launch(c, GID_KIND_APPLY,
         [&] { GID_DISPATCH(c, apply, c, 1, 0, 1, (const float*)c->pA, (float*)nullptr, c->pB); });
  if (int rc = check_launch(c, "k_apply")) return rc;
  return from_pitched(c, q_dev, c->pB);
}

extern "C" int gid_stage_pcg(gid_ctx* c, int m_inner, float* delta_dev) {
  if (!c || !delta_dev || m_inner < 1) return fail(c, GID_ERR_INVALID_ARG, "bad argument");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "no frame/state");
  if (int rc = enqueue_gn_step(c, m_inner, 2)) return rc;
  return from_pitched(c, delta_dev, c->d);
}

extern "C" int gid_stage_dense_normal(gid_ctx* c, double* A_host, double* g_host) {
  if (!c || !A_host || !g_host) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "no frame/state");
  launch(c, GID_KIND_DENSE, [&] { GID_DISPATCH(c, dense, c, 0); });
  if (int rc = check_launch(c, "k_dense")) return rc;
  GID_TRY_CUDA(c, cudaMemcpyAsync(A_host, c->sc->A, sizeof(double) * 3 * c->K * c->K, cudaMemcpyDeviceToHost,
                                  c->stream));
  GID_TRY_CUDA(c, cudaMemcpyAsync(g_host, c->sc->g, sizeof(double) * 3 * c->K, cudaMemcpyDeviceToHost, c->stream));
  return sync_status(c);
}

// ---------------------------------------------------------------- counters

extern "C" int gid_launch_count(const gid_ctx* c, long long* n) {
  if (!c || !n) return GID_ERR_INVALID_ARG;
  *n = c->launches;
  return GID_OK;
}

extern "C" int gid_profile(gid_ctx* c, int enable) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (enable && c->ev.empty()) {
    c->ev.resize(16384 + 1);
    for (auto& e : c->ev) GID_TRY_CUDA(c, cudaEventCreate(&e));
  }
  c->prof = enable != 0;
  return GID_OK;
}

extern "C" int gid_profile_read(gid_ctx* c, double* ms, long long* count) {
  if (!c || !ms || !count) return fail(c, GID_ERR_INVALID_ARG, "NULL argument");
  GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < c->ev_kind.size(); i++) {
    float t = 0.f;
    GID_TRY_CUDA(c, cudaEventElapsedTime(&t, c->ev[i], c->ev[i + 1]));
    c->prof_ms[c->ev_kind[i]] += t;
    c->prof_n[c->ev_kind[i]]++;
  }
  c->ev_kind.clear();
  for (int k = 0; k < GID_NUM_KINDS; k++) {
    ms[k] = c->prof_ms[k];
    count[k] = c->prof_n[k];
    c->prof_ms[k] = 0;
    c->prof_n[k] = 0;
  }
  return GID_OK;
}

// ---------------------------------------------------------------- operator tile shape

// Plans the resident PCG kernel for the context's frame (once) and allocates
// its exchange buffers on first use.  GID_ERR_INVALID_ARG if it does not fit.
static int res_prepare(gid_ctx* c) {
  if (!c->res_planned) GID_DISPATCH(c, res_plan, c);
  if (c->res_blocks <= 0)
    return fail(c, GID_ERR_INVALID_ARG,
                "the resident PCG kernel does not fit this frame on this device (its tiles of the PCG state "
                "exceed one block per SM)");
  if (!c->zx) {
    // the coefficient planes as a 3-D tensor (columns, rows, planes); one box is
    // one plane of a tile with the row above and 4 columns to the left
    auto fn = encode_fn();
    const int nc = coef_planes(c->K, c->w.n_spatial_pairs);
    const cuuint64_t dims[3] = {(cuuint64_t)c->pitch, (cuuint64_t)c->H, (cuuint64_t)nc};
    const cuuint64_t strides[2] = {(cuuint64_t)c->pitch * sizeof(float), (cuuint64_t)c->plane * sizeof(float)};
    const cuuint32_t box[3] = {(cuuint32_t)(4 * c->res.TX + 8), (cuuint32_t)(c->res.TH + 1), 1u};
    const cuuint32_t es[3] = {1u, 1u, 1u};
    if (!fn || fn(&c->res_map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c->coef, dims, strides, box, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return fail(c, GID_ERR_CUDA, "cuTensorMapEncodeTiled failed for the resident coefficient stream");
  }
  if (!c->zx) {
    const size_t zb = 2 * (size_t)c->V * c->plane * sizeof(float);
    const size_t xb = (size_t)RES_ROWS * RES_NV * RES_MAXB * sizeof(double) + RES_ROWS * 128;
    if (cudaMalloc(&c->zx, zb) != cudaSuccess || cudaMalloc(&c->xval, xb) != cudaSuccess) {
      cudaGetLastError();
      cudaFree(c->zx);
      cudaFree(c->xval);
      c->zx = nullptr;
      c->xval = nullptr;
      return fail(c, GID_ERR_OOM, "resident PCG exchange buffers");
    }
    // the exchange planes' padding columns and unowned chunks read as zero; the
    // all-reduce counters are cleared by every linearisation
    GID_TRY_CUDA(c, cudaMemsetAsync(c->zx, 0, zb, c->stream));
    GID_TRY_CUDA(c, cudaMemsetAsync(c->xval, 0, xb, c->stream));
    GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  }
  return GID_OK;
}

// The fused PCG step's odd-step buffers (allocated once, zeroed: their padding
// columns stay zero like those of every PCG vector).
static int fused_prepare(gid_ctx* c) {
  if (c->fbuf) return GID_OK;
  const size_t bytes = sizeof(float) * 2 * (size_t)c->V * c->plane;
  if (cudaMalloc(&c->fbuf, bytes) != cudaSuccess) {
    cudaGetLastError();
    c->fbuf = nullptr;
    return fail(c, GID_ERR_OOM, "cudaMalloc of the fused PCG step's buffers");
  }
  GID_TRY_CUDA(c, cudaMemsetAsync(c->fbuf, 0, bytes, c->stream));
  return GID_OK;
}

extern "C" int gid_set_apply_tile(gid_ctx* c, int rows) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (rows == GID_PCG_RESIDENT) {
    if (int rc = res_prepare(c)) return rc;
    c->resident = true;
    c->persistent = false;
    return GID_OK;
  }
  if (rows == 0) {
    if (c->pcg_blocks <= 0) return fail(c, GID_ERR_INVALID_ARG, "the persistent PCG kernel cannot run on this device");
    c->persistent = true;
    c->resident = false;
    return GID_OK;
  }
  const bool fused = rows > 0 && (rows & GID_PCG_FUSED);
  if (fused) rows &= ~GID_PCG_FUSED;
  if ((rows != 2 && rows != 4 && rows != 8 && rows != 16 && rows != 17) || (fused && rows == 16))
    return fail(c, GID_ERR_INVALID_ARG,
                "tile rows must be -1 (resident), 0 (persistent), 2, 4, 8, 16 or 17 (2, 4, 8 or 17 | GID_PCG_FUSED)");
  if (fused)
    if (int rc = fused_prepare(c)) return rc;
  c->apply_th = rows;
  c->persistent = false;
  c->resident = false;
  c->fused = fused;
  return GID_OK;
}

extern "C" int gid_get_pcg_layout(gid_ctx* c, int* rows, int* tile_w, int* tile_h, int* blocks) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  const int k = pcg_kernel(c);
  if (rows) *rows = k == 2 ? GID_PCG_RESIDENT : (k == 1 ? 0 : (k == 3 ? c->apply_th | GID_PCG_FUSED : c->apply_th));
  if (!c->res_planned) GID_DISPATCH(c, res_plan, c);
  if (tile_w) *tile_w = c->res_blocks > 0 ? 4 * c->res.TX : 0;
  if (tile_h) *tile_h = c->res_blocks > 0 ? c->res.TH : 0;
  if (blocks) *blocks = c->res_blocks;
  return GID_OK;
}

// ---------------------------------------------------------------- L2 persistence of the coefficients

// Contexts of this process whose launches carry a window (the set-aside is
// released when the last one turns it off or is destroyed); the count and the
// device limit are changed under one lock.
static int g_l2_users = 0;
static std::mutex g_l2_mu;

static void l2_release(gid_ctx* c) {
  if (!c->l2_window) return;
  std::lock_guard<std::mutex> lock(g_l2_mu);
  c->l2_window = false;
  if (--g_l2_users == 0) {
    cudaCtxResetPersistingL2Cache();
    cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, 0);
    cudaGetLastError();
  }
}

extern "C" int gid_get_l2_window(const gid_ctx* c) { return c ? (c->l2_window ? 1 : 0) : -1; }

extern "C" int gid_set_l2_window(gid_ctx* c, int on) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if ((on != 0) == c->l2_window) return GID_OK;
  // the cached graphs hold launches with the other attribute set
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gs) cudaStreamSynchronize(c->gs);
  for (auto& gr : c->graphs) cudaGraphExecDestroy(gr.exec);
  c->graphs.clear();
  if (!on) {
    l2_release(c);
    return GID_OK;
  }
  int dev = 0, maxp = 0, maxw = 0;
  GID_TRY_CUDA(c, cudaGetDevice(&dev));
  GID_TRY_CUDA(c, cudaDeviceGetAttribute(&maxp, cudaDevAttrMaxPersistingL2CacheSize, dev));
  GID_TRY_CUDA(c, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxAccessPolicyWindowSize, dev));
  if (maxp <= 0 || maxw <= 0) return fail(c, GID_ERR_INVALID_ARG, "no persisting L2 on this device");
  // the coefficients and as many of q, p and z (allocated just before them, in that
  // order backwards) as fit; a window the set-aside cannot hold whole thrashes it
  // (measured slower than none)
  const char* coef_end = reinterpret_cast<const char*>(c->coef) +
                         sizeof(float) * (size_t)coef_planes(c->K, c->w.n_spatial_pairs) * c->plane;
  const float* starts[4] = {c->z, c->pA, c->q, c->coef};  // consecutive in the pool
  const char* base = nullptr;
  size_t win = 0;
  for (const float* s0 : starts) {
    base = reinterpret_cast<const char*>(s0);
    win = (size_t)(coef_end - base);
    if (win <= (size_t)maxp && win <= (size_t)maxw) break;
  }
  if (win > (size_t)maxp || win > (size_t)maxw)
    return fail(c, GID_ERR_INVALID_ARG, "the coefficient planes exceed the device's persisting L2");
  std::lock_guard<std::mutex> lock(g_l2_mu);
  size_t cur = 0;
  GID_TRY_CUDA(c, cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  const size_t want = std::min(win, (size_t)maxp);
  if (cur < want) GID_TRY_CUDA(c, cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want));
  GID_TRY_CUDA(c, cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize));
  c->l2win.base_ptr = const_cast<char*>(base);
  c->l2win.num_bytes = win;
  c->l2win.hitRatio = std::min(1.0f, (float)cur / (float)win);
  c->l2win.hitProp = cudaAccessPropertyPersisting;
  c->l2win.missProp = cudaAccessPropertyStreaming;
  c->l2_window = true;
  g_l2_users++;
  return GID_OK;
}

// ---------------------------------------------------------------- PCG history

extern "C" int gid_set_pcg_history(gid_ctx* c, int on) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if ((on != 0) == c->record_rho) return GID_OK;
  // the cached graphs hold the other launch sequence
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gs) cudaStreamSynchronize(c->gs);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  c->record_rho = on != 0;
  return GID_OK;
}

extern "C" int gid_pcg_history(gid_ctx* c, double* rho_host, int max_n, int* n_out) {
  if (!c || !rho_host || !n_out || max_n < 0) return fail(c, GID_ERR_INVALID_ARG, "bad argument");
  const int n = c->hist_valid ? std::min({c->last_m_inner, PCG_HIST, max_n}) : 0;
  *n_out = n;
  if (n > 0)
    GID_TRY_CUDA(c, cudaMemcpyAsync(rho_host, c->sc->rho_hist, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  return sync_status(c);
}

// ---------------------------------------------------------------- fault injection (tests)

extern "C" int gid_debug_inject(gid_ctx* c, int phantom_blocks, long long spin_limit) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (phantom_blocks < 0 || spin_limit < 0) return fail(c, GID_ERR_INVALID_ARG, "phantom_blocks, spin_limit >= 0");
  struct {
    unsigned int phantom;
    long long spin_limit;
  } v = {(unsigned int)phantom_blocks, spin_limit};
  GID_TRY_CUDA(c, cudaMemcpyAsync(&c->sc->phantom, &v.phantom, sizeof(v.phantom), cudaMemcpyHostToDevice, c->stream));
  GID_TRY_CUDA(c, cudaMemcpyAsync(&c->sc->spin_limit, &v.spin_limit, sizeof(v.spin_limit), cudaMemcpyHostToDevice,
                                  c->stream));
  GID_TRY_CUDA(c, cudaStreamSynchronize(c->stream));
  return GID_OK;
}

// ---------------------------------------------------------------- preconditioner

extern "C" int gid_set_preconditioner(gid_ctx* c, int kind) {
  if (!c) return fail(c, GID_ERR_INVALID_ARG, "NULL ctx");
  if (kind != GID_PRECOND_JACOBI && kind != GID_PRECOND_BLOCK)
    return fail(c, GID_ERR_INVALID_ARG, "preconditioner must be GID_PRECOND_JACOBI or GID_PRECOND_BLOCK");
  if (kind == c->precond) return GID_OK;
  if (kind == GID_PRECOND_BLOCK && !c->blk) {
    const size_t nb = (size_t)block_planes(c->K);
    if (cudaMalloc(&c->blk, nb * c->plane * sizeof(float)) != cudaSuccess) {
      cudaGetLastError();
      c->blk = nullptr;
      return fail(c, GID_ERR_OOM, "block-Jacobi factor planes");
    }
    int cap = 0;
    switch (c->K) {
      case 1: cap = Launch<1>::block_capacity(c); break;
      case 2: cap = Launch<2>::block_capacity(c); break;
      case 3: cap = Launch<3>::block_capacity(c); break;
      case 4: cap = Launch<4>::block_capacity(c); break;
      case 5: cap = Launch<5>::block_capacity(c); break;
      case 6: cap = Launch<6>::block_capacity(c); break;
      case 7: cap = Launch<7>::block_capacity(c); break;
      case 8: cap = Launch<8>::block_capacity(c); break;
      case 9: cap = Launch<9>::block_capacity(c); break;
      default: cap = Launch<10>::block_capacity(c); break;
    }
    // one pixel per thread; never more blocks than the partial slots hold
    const long want = (c->plane + 255) / 256;
    c->blk_blocks = (int)std::max(1L, std::min({want, (long)cap, (long)c->nbmax}));
  }
  // the cached graphs hold the other preconditioner's launch sequence
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->gs) cudaStreamSynchronize(c->gs);
  for (auto& g : c->graphs) cudaGraphExecDestroy(g.exec);
  c->graphs.clear();
  c->precond = kind;
  return GID_OK;
}

extern "C" int gid_get_preconditioner(const gid_ctx* c) { return c ? c->precond : -1; }

extern "C" int gid_autotune(gid_ctx* c, int reps, int* rows_out, float* us_out) {
  if (!c || reps < 1) return fail(c, GID_ERR_INVALID_ARG, "bad argument");
  if (!c->has_frame || !c->initialised) return fail(c, GID_ERR_STATE, "autotune needs a frame and a state");
  // A PCG start at the current state, then timed (operator step + vector step)
  // pairs: the in-loop cost, cache interference included.  The PCG vectors and
  // scalars it touches are re-initialised by the next Gauss-Newton step; X is
  // not modified.
  launch(c, GID_KIND_LINEARIZE, [&] { GID_DISPATCH(c, linearize, c, 0, (float*)nullptr, (float*)nullptr); });
  if (int rc = check_launch(c, "k_linearize")) return rc;
  cudaEvent_t e0, e1;
  GID_TRY_CUDA(c, cudaEventCreate(&e0));
  GID_TRY_CUDA(c, cudaEventCreate(&e1));
  // the two-kernel loop's tile shapes and their slots in us_out (16 rows came last)
  const int cand[4] = {2, 4, 8, 17}, tiled[5] = {2, 4, 8, 17, 16}, slot[5] = {0, 1, 2, 3, 10};
  float best = 1e30f;
  int best_th = c->apply_th;
  c->persistent = false;
  c->resident = false;
  c->fused = false;
  for (int i = 0; i < 5; i++) {
    c->apply_th = tiled[i];
    int it = 0;
    auto pair = [&](int first) {
      ++it;
      GID_DISPATCH(c, apply, c, 0, first, it, (const float*)c->pA, c->pA, c->q);
      GID_DISPATCH(c, update, c, it, (const float*)c->pA, 0);
    };
    GID_DISPATCH(c, linearize, c, 0, (float*)nullptr, (float*)nullptr);
    pair(1);
    pair(0);
    cudaEventRecord(e0, c->stream);
    for (int r = 0; r < reps; r++) pair(0);
    cudaEventRecord(e1, c->stream);
    c->launches += 2 * (reps + 2);
    if (int rc = check_launch(c, "k_apply")) return rc;
    GID_TRY_CUDA(c, cudaEventSynchronize(e1));
    float ms = 0.f;
    GID_TRY_CUDA(c, cudaEventElapsedTime(&ms, e0, e1));
    const float us = 1000.f * ms / reps;
    if (us_out) us_out[slot[i]] = us;
    if (us < best) {
      best = us;
      best_th = tiled[i];
    }
  }
  c->apply_th = best_th;
  // the single-launch loops (persistent, resident): the time of a Gauss-Newton
  // step of reps + 2 PCG steps less that of one of 2, per PCG step (the
  // linearisation and the launch cancel)
  auto time_loop = [&](float* us) -> int {
    float ms[2] = {0.f, 0.f};
    for (int i = 0; i < 2; i++) {
      cudaEventRecord(e0, c->stream);
      if (int rc = enqueue_gn_step(c, i == 0 ? 2 : reps + 2, 2)) return rc;
      cudaEventRecord(e1, c->stream);
      GID_TRY_CUDA(c, cudaEventSynchronize(e1));
      GID_TRY_CUDA(c, cudaEventElapsedTime(&ms[i], e0, e1));
    }
    *us = 1000.f * (ms[1] - ms[0]) / reps;
    return sync_status(c);
  };
  int choice = best_th;  // rows, 0 persistent, GID_PCG_RESIDENT resident, rows | GID_PCG_FUSED
  c->resident = false;
  c->fused = false;
  if (c->pcg_blocks > 0) {
    c->persistent = true;
    float us = 0.f;
    if (int rc = time_loop(&us)) return rc;
    if (us_out) us_out[4] = us;
    if (us < best) {
      best = us;
      choice = 0;
    }
    c->persistent = false;
  } else if (us_out) {
    us_out[4] = -1.f;
  }
  if (c->precond == GID_PRECOND_JACOBI && res_prepare(c) == GID_OK) {
    c->resident = true;
    float us = 0.f;
    if (int rc = time_loop(&us)) return rc;
    if (us_out) us_out[5] = us;
    if (us < best) {
      best = us;
      choice = GID_PCG_RESIDENT;
    }
    c->resident = false;
  } else if (us_out) {
    us_out[5] = -1.f;
  }
  // the fused step (one kernel per PCG step) with each tile shape
  const int th_tiled = c->apply_th;
  for (int i = 0; i < 4; i++) {
    if (c->precond != GID_PRECOND_JACOBI || fused_prepare(c) != GID_OK) {
      if (us_out) us_out[6 + i] = -1.f;
      continue;
    }
    c->fused = true;
    c->apply_th = cand[i];
    float us = 0.f;
    if (int rc = time_loop(&us)) return rc;
    if (us_out) us_out[6 + i] = us;
    if (us < best) {
      best = us;
      choice = cand[i] | GID_PCG_FUSED;
    }
  }
  c->fused = choice > 0 && (choice & GID_PCG_FUSED);
  c->apply_th = c->fused ? (choice & ~GID_PCG_FUSED) : th_tiled;
  c->persistent = choice == 0;
  c->resident = choice == GID_PCG_RESIDENT;
  // the chosen loop with and without the L2 window over the coefficients (where
  // they fit in the persisting set-aside): keep the faster
  const bool had_window = c->l2_window;
  if (gid_set_l2_window(c, 0) == GID_OK && gid_set_l2_window(c, 1) == GID_OK) {
    float with = 0.f, without = 0.f;
    if (int rc = time_loop(&with)) return rc;
    gid_set_l2_window(c, 0);
    if (int rc = time_loop(&without)) return rc;
    if (with < without) gid_set_l2_window(c, 1);
  } else {
    c->err.clear();
    gid_set_l2_window(c, had_window ? 1 : 0);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rows_out) *rows_out = choice;
  return GID_OK;
}

// ---------------------------------------------------------------- batches of videos

struct gid_batch {
  int n = 0;
  std::vector<gid_ctx*> ctx;
  std::vector<cudaStream_t> streams;  // one per video; the contexts run on these
  cudaStream_t user = nullptr;        // the caller's stream
  cudaStream_t bs = nullptr;          // capture / replay stream of the batch graph
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  std::vector<cudaEvent_t> ev_join;
  struct Graph {
    std::string key;
    cudaGraphExec_t exec;
    long long kernels;
    std::vector<void*> tables;  // device work-list tables the graph's launches read
  };
  std::vector<Graph> graphs;
  bool worklist = true;  // PCG steps as work-list launches per K (gid_batch_set_worklist)
  bool persistent_wl = false;  // ... as one cooperative launch per K and Gauss-Newton step
  std::string err;
};

static std::string g_batch_err;

static int bfail(gid_batch* b, int code, const std::string& m) {
  if (b)
    b->err = m;
  else
    g_batch_err = m;
  return code;
}

#define GID_BTRY(b, call)                                                                          \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return bfail((b), GID_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" void gid_batch_destroy(gid_batch* b) {
  if (!b) return;
  for (auto* c : b->ctx) {
    if (!c) continue;
    cudaStreamSynchronize(c->stream);
    gid_destroy(c);
  }
  if (b->bs) cudaStreamSynchronize(b->bs);
  for (auto& g : b->graphs) {
    cudaGraphExecDestroy(g.exec);
    for (void* p : g.tables) cudaFree(p);
  }
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->ev_join) cudaEventDestroy(e);
  if (b->bs) cudaStreamDestroy(b->bs);
  if (b->ev_in) cudaEventDestroy(b->ev_in);
  if (b->ev_out) cudaEventDestroy(b->ev_out);
  delete b;
}

extern "C" int gid_batch_create(int n, const int* H, const int* W, const int* K, const gid_weights* w, int per_video,
                                void* stream, gid_batch** out) {
  if (!out || n < 1 || !H || !W || !K) return bfail(nullptr, GID_ERR_INVALID_ARG, "bad arguments");
  *out = nullptr;
  gid_batch* b = new (std::nothrow) gid_batch();
  if (!b) return bfail(nullptr, GID_ERR_OOM, "host allocation");
  b->n = n;
  b->user = (cudaStream_t)stream;
  b->ctx.assign(n, nullptr);
  auto bail = [&](int rc, const std::string& m) {
    gid_batch_destroy(b);
    return bfail(nullptr, rc, m);
  };
  if (cudaStreamCreateWithFlags(&b->bs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming) != cudaSuccess)
    return bail(GID_ERR_CUDA, "batch stream / events");
  for (int i = 0; i < n; i++) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(GID_ERR_CUDA, "stream");
    b->streams.push_back(s);
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return bail(GID_ERR_CUDA, "event");
    b->ev_join.push_back(e);
    int rc = gid_create(H[i], W[i], K[i], w ? (per_video ? &w[i] : w) : nullptr, s, &b->ctx[i]);
    if (rc) return bail(rc, std::string("video ") + std::to_string(i) + ": " + gid_last_error(nullptr));
  }
  *out = b;
  return GID_OK;
}

extern "C" const char* gid_batch_last_error(const gid_batch* b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

extern "C" gid_ctx* gid_batch_ctx(gid_batch* b, int i) { return (b && i >= 0 && i < b->n) ? b->ctx[i] : nullptr; }

// Order the video streams after the caller's stream (before per-video work).
static int batch_fence_in(gid_batch* b) {
  GID_BTRY(b, cudaEventRecord(b->ev_in, b->user));
  for (int i = 0; i < b->n; i++) GID_BTRY(b, cudaStreamWaitEvent(b->streams[i], b->ev_in, 0));
  return GID_OK;
}

// Order the caller's stream after every video stream.
static int batch_fence_out(gid_batch* b) {
  for (int i = 0; i < b->n; i++) {
    GID_BTRY(b, cudaEventRecord(b->ev_join[i], b->streams[i]));
    GID_BTRY(b, cudaStreamWaitEvent(b->user, b->ev_join[i], 0));
  }
  return GID_OK;
}

extern "C" int gid_batch_set_frames(gid_batch* b, const float* const* rgb_dev, const uint8_t* const* labels_dev) {
  if (!b || !rgb_dev || !labels_dev) return bfail(b, GID_ERR_INVALID_ARG, "NULL argument");
  if (int rc = batch_fence_in(b)) return rc;
  for (int i = 0; i < b->n; i++)
    if (int rc = gid_set_frame(b->ctx[i], rgb_dev[i], labels_dev[i]))
      return bfail(b, rc, std::string("video ") + std::to_string(i) + ": " + gid_last_error(b->ctx[i]));
  return batch_fence_out(b);
}

extern "C" int gid_batch_init(gid_batch* b, int mode) {
  if (!b) return bfail(b, GID_ERR_INVALID_ARG, "NULL batch");
  if (int rc = batch_fence_in(b)) return rc;
  for (int i = 0; i < b->n; i++)
    if (int rc = gid_init(b->ctx[i], mode))
      return bfail(b, rc, std::string("video ") + std::to_string(i) + ": " + gid_last_error(b->ctx[i]));
  return batch_fence_out(b);
}

extern "C" int gid_batch_new_sequence(gid_batch* b) {
  if (!b) return bfail(b, GID_ERR_INVALID_ARG, "NULL batch");
  if (int rc = batch_fence_in(b)) return rc;
  for (int i = 0; i < b->n; i++)
    if (int rc = gid_new_sequence(b->ctx[i])) return bfail(b, rc, gid_last_error(b->ctx[i]));
  return batch_fence_out(b);
}

// One graph per batch configuration: every video's run is a branch forked from
// and joined to the batch stream, so the whole frame-step of all videos is one
// graph launch and the videos' kernels run concurrently.
// The work-list form of a batch's run, enqueued for capture on b->bs: per
// The videos of a batch that share K, with their work-list tables.
struct WorkGroup {
  int K;
  std::vector<int> vid;
  MultiVideo* dv = nullptr;
  CUtensorMap* dm = nullptr;
  int tiles = 0, upd = 0;
  int coop = 0;  // co-resident blocks of the persistent form (0: not available)
};

// The device tables of the work-list launches (made before the capture: the
// allocation and the copies are not capturable).  False on a CUDA error.
static bool build_worklist(gid_batch* b, std::vector<WorkGroup>& groups, std::vector<void*>& tables) {
  constexpr int TH = WL_TH;
  using Group = WorkGroup;
  for (int i = 0; i < b->n; i++) {
    Group* gp = nullptr;
    for (auto& gr : groups)
      if (gr.K == b->ctx[i]->K) gp = &gr;
    if (!gp) {
      groups.push_back(Group{b->ctx[i]->K, {}});
      gp = &groups.back();
    }
    gp->vid.push_back(i);
  }
  for (auto& gr : groups) {
    const int nv = (int)gr.vid.size();
    std::vector<MultiVideo> hv(nv);
    std::vector<CUtensorMap> hm(2 * nv);
    long total_items = 0;
    for (int v = 0; v < nv; v++) total_items += (long)b->ctx[gr.vid[v]]->V * (b->ctx[gr.vid[v]]->plane / 4);
    const int wave = b->ctx[gr.vid[0]]->upd_cap;
    for (int v = 0; v < nv; v++) {
      gid_ctx* c = b->ctx[gr.vid[v]];
      const gid_ctx::Maps* m = tile_maps(c, c->z, TH);
      if (!m) return false;
      hm[2 * v] = m->r;
      hm[2 * v + 1] = m->t;
      MultiVideo& mv = hv[v];
      memset(&mv, 0, sizeof(mv));
      mv.P = params(c);
      mv.p = c->pA;
      mv.ntx = (c->W + VTW - 1) / VTW;
      mv.ntiles = mv.ntx * ((c->H + TH - 1) / TH);
      const long items = (long)c->V * (c->plane / 4);
      mv.nupd = (int)std::max(1L, std::min({(long)std::lround((double)wave * items / total_items), (items + 255) / 256,
                                            (long)c->nbmax}));
      mv.tile0 = gr.tiles;
      mv.upd0 = gr.upd;
      gr.tiles += mv.ntiles;
      gr.upd += mv.nupd;
    }
    if (b->persistent_wl) {
      switch (gr.K) {
        case 1: gr.coop = Launch<1>::pcg_multi_capacity(); break;
        case 2: gr.coop = Launch<2>::pcg_multi_capacity(); break;
        case 3: gr.coop = Launch<3>::pcg_multi_capacity(); break;
        case 4: gr.coop = Launch<4>::pcg_multi_capacity(); break;
        case 5: gr.coop = Launch<5>::pcg_multi_capacity(); break;
        case 6: gr.coop = Launch<6>::pcg_multi_capacity(); break;
        case 7: gr.coop = Launch<7>::pcg_multi_capacity(); break;
        case 8: gr.coop = Launch<8>::pcg_multi_capacity(); break;
        case 9: gr.coop = Launch<9>::pcg_multi_capacity(); break;
        default: gr.coop = Launch<10>::pcg_multi_capacity(); break;
      }
      if (gr.coop <= 0) return false;
    }
    if (cudaMalloc(&gr.dv, sizeof(MultiVideo) * nv) != cudaSuccess) return false;
    tables.push_back(gr.dv);
    if (cudaMalloc(&gr.dm, sizeof(CUtensorMap) * 2 * nv) != cudaSuccess) return false;
    tables.push_back(gr.dm);
    if (cudaMemcpy(gr.dv, hv.data(), sizeof(MultiVideo) * nv, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(gr.dm, hm.data(), sizeof(CUtensorMap) * 2 * nv, cudaMemcpyHostToDevice) != cudaSuccess)
      return false;
  }
  return true;
}

static void enqueue_apply_multi(gid_batch* b, const WorkGroup& gr, int m) {
  const int nv = (int)gr.vid.size(), first = m == 1 ? 1 : 0;
  switch (gr.K) {
    case 1: Launch<1>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 2: Launch<2>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 3: Launch<3>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 4: Launch<4>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 5: Launch<5>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 6: Launch<6>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 7: Launch<7>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 8: Launch<8>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    case 9: Launch<9>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
    default: Launch<10>::apply_multi(b->bs, gr.dv, nv, gr.dm, first, m, gr.tiles); break;
  }
}

static void enqueue_update_multi(gid_batch* b, const WorkGroup& gr, int m, int last) {
  switch (gr.K) {
    case 1: Launch<1>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 2: Launch<2>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 3: Launch<3>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 4: Launch<4>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 5: Launch<5>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 6: Launch<6>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 7: Launch<7>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 8: Launch<8>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    case 9: Launch<9>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
    default: Launch<10>::update_multi(b->bs, gr.dv, (int)gr.vid.size(), m, last, gr.upd); break;
  }
}

// Per Gauss-Newton step every video's linearisation on its own stream, then M
// PCG steps as one operator launch and one vector launch per K over all videos
// with that K (k_apply_multi / k_update_multi, operator tiles of 128 x WL_TH,
// about one wave of vector blocks per launch split by plane size), then every
// video's base-colour step on its own stream.  Returns the kernels enqueued,
// < 0 on error.
static long long enqueue_worklist(gid_batch* b, std::vector<WorkGroup>& groups, int n_outer, int m_inner,
                                  const std::vector<int>& refine) {
  long long kernels = 0;
  auto fork_join = [&](auto enqueue_one) -> bool {
    if (cudaEventRecord(b->ev_in, b->bs) != cudaSuccess) return false;
    for (int i = 0; i < b->n; i++) {
      gid_ctx* c = b->ctx[i];
      if (cudaStreamWaitEvent(b->streams[i], b->ev_in, 0) != cudaSuccess) return false;
      kernels += enqueue_one(c, i);
      if (cudaEventRecord(b->ev_join[i], b->streams[i]) != cudaSuccess ||
          cudaStreamWaitEvent(b->bs, b->ev_join[i], 0) != cudaSuccess)
        return false;
    }
    return true;
  };
  for (int n = 0; n < n_outer; n++) {
    bool ok = fork_join([&](gid_ctx* c, int) -> long long {
      c->last_m_inner = m_inner;
      c->hist_valid = false;
      GID_DISPATCH(c, linearize, c, 0, (float*)nullptr, (float*)nullptr);
      return 1;
    });
    if (!ok) return -1;
    if (b->persistent_wl) {
      for (auto& gr : groups) {
        DevScalars* bar = b->ctx[gr.vid[0]]->sc;
        const int nv = (int)gr.vid.size();
        cudaError_t e = cudaSuccess;
        switch (gr.K) {
          case 1: e = Launch<1>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 2: e = Launch<2>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 3: e = Launch<3>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 4: e = Launch<4>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 5: e = Launch<5>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 6: e = Launch<6>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 7: e = Launch<7>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 8: e = Launch<8>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          case 9: e = Launch<9>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
          default: e = Launch<10>::pcg_multi(b->bs, gr.dv, nv, gr.dm, gr.tiles, gr.upd, m_inner, bar, gr.coop); break;
        }
        if (e != cudaSuccess) return -1;
        kernels++;
      }
    }
    for (int m = 1; m <= m_inner && !b->persistent_wl; m++) {
      for (auto& gr : groups) {
        enqueue_apply_multi(b, gr, m);
        kernels++;
      }
      for (auto& gr : groups) {
        enqueue_update_multi(b, gr, m, m == m_inner ? 1 : 0);
        kernels++;
      }
    }
    ok = fork_join([&](gid_ctx* c, int i) -> long long {
      if (!refine[i]) return 0;
      GID_DISPATCH(c, dense, c, 1);
      return 1;
    });
    if (!ok) return -1;
  }
  return cudaGetLastError() == cudaSuccess ? kernels : -1;
}

extern "C" int gid_batch_set_worklist(gid_batch* b, int on) {
  if (!b) return bfail(b, GID_ERR_INVALID_ARG, "NULL batch");
  b->worklist = on != 0;
  b->persistent_wl = on == 2;
  return GID_OK;
}

extern "C" int gid_batch_run(gid_batch* b, int n_outer, int m_inner) {
  gid::NvtxRange nvtx_range("gid_batch_run");
  if (!b) return bfail(b, GID_ERR_INVALID_ARG, "NULL batch");
  if (n_outer < 1 || m_inner < 1) return bfail(b, GID_ERR_INVALID_ARG, "n_outer >= 1 and m_inner >= 1");
  // the work-list form needs Jacobi PCG in every video
  bool wl = b->worklist;
  for (int i = 0; i < b->n; i++) wl = wl && b->ctx[i]->precond == GID_PRECOND_JACOBI;
  std::string key = std::to_string(n_outer) + "," + std::to_string(m_inner) + (wl ? (b->persistent_wl ? ",p" : ",w") : ",b");
  std::vector<int> refine(b->n);
  for (int i = 0; i < b->n; i++) {
    gid_ctx* c = b->ctx[i];
    if (!c->has_frame || !c->initialised) return bfail(b, GID_ERR_STATE, "gid_batch_run before frames / init");
    c->persistent = false;  // concurrent cooperative grids could not all be co-resident
    refine[i] = c->w.refine_base_colors == 1 || (c->w.refine_base_colors == 2 && c->frames_solved == 0);
    key += ";" + std::to_string(refine[i]) + std::to_string((int)c->temporal_active) + std::to_string(c->apply_th);
  }
  gid_batch::Graph* g = nullptr;
  for (auto& e : b->graphs)
    if (e.key == key) g = &e;
  if (!g) {
    long long kernels = 0;
    std::vector<void*> tables;
    std::vector<WorkGroup> groups;
    if (wl && !build_worklist(b, groups, tables)) {
      cudaGetLastError();
      for (void* p : tables) cudaFree(p);
      return bfail(b, GID_ERR_CUDA,
                   b->persistent_wl ? "batch work-list tables, or the persistent work list cannot be co-scheduled"
                                    : "batch work-list tables");
    }
    GID_BTRY(b, cudaStreamBeginCapture(b->bs, cudaStreamCaptureModeThreadLocal));
    int rc = GID_OK;
    if (cudaEventRecord(b->ev_in, b->bs) != cudaSuccess) rc = GID_ERR_CUDA;
    if (wl && !rc) {
      kernels = enqueue_worklist(b, groups, n_outer, m_inner, refine);
      if (kernels < 0) rc = GID_ERR_CUDA;
    }
    for (int i = 0; i < b->n && !rc && !wl; i++) {
      gid_ctx* c = b->ctx[i];
      if (cudaStreamWaitEvent(b->streams[i], b->ev_in, 0) != cudaSuccess) {
        rc = GID_ERR_CUDA;
        break;
      }
      const long long l0 = c->launches;
      rc = enqueue_run(c, n_outer, m_inner, refine[i]);
      kernels += c->launches - l0;
      c->launches = l0;
      if (!rc && (cudaEventRecord(b->ev_join[i], b->streams[i]) != cudaSuccess ||
                  cudaStreamWaitEvent(b->bs, b->ev_join[i], 0) != cudaSuccess))
        rc = GID_ERR_CUDA;
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->bs, &graph);
    if (rc || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      for (void* p : tables) cudaFree(p);
      return bfail(b, rc ? rc : GID_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e));
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      for (void* p : tables) cudaFree(p);
      return bfail(b, GID_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
    b->graphs.push_back({key, exec, kernels, tables});
    g = &b->graphs.back();
  }
  // replay after everything already queued for the videos and the caller
  for (int i = 0; i < b->n; i++) {
    GID_BTRY(b, cudaEventRecord(b->ev_join[i], b->streams[i]));
    GID_BTRY(b, cudaStreamWaitEvent(b->bs, b->ev_join[i], 0));
  }
  GID_BTRY(b, cudaEventRecord(b->ev_in, b->user));
  GID_BTRY(b, cudaStreamWaitEvent(b->bs, b->ev_in, 0));
  GID_BTRY(b, cudaGraphLaunch(g->exec, b->bs));
  GID_BTRY(b, cudaEventRecord(b->ev_out, b->bs));
  GID_BTRY(b, cudaStreamWaitEvent(b->user, b->ev_out, 0));
  for (int i = 0; i < b->n; i++) GID_BTRY(b, cudaStreamWaitEvent(b->streams[i], b->ev_out, 0));
  long long per_video = g->kernels / b->n;  // bookkeeping only: split the count evenly
  for (int i = 0; i < b->n; i++) {
    b->ctx[i]->launches += (i == 0) ? g->kernels - per_video * (b->n - 1) : per_video;
    b->ctx[i]->frames_solved++;
  }
  return GID_OK;
}

// Tile-shape cache: one line "H W K rows" per frame shape.
static void read_tile_cache(const char* path, std::vector<std::array<int, 4>>& rows) {
  FILE* f = path ? fopen(path, "r") : nullptr;
  if (!f) return;
  std::array<int, 4> r;
  while (fscanf(f, "%d %d %d %d", &r[0], &r[1], &r[2], &r[3]) == 4) rows.push_back(r);
  fclose(f);
}

extern "C" int gid_batch_autotune(gid_batch* b, const char* cache_path, int reps) {
  if (!b || reps < 1) return bfail(b, GID_ERR_INVALID_ARG, "bad argument");
  std::vector<std::array<int, 4>> cache;
  read_tile_cache(cache_path, cache);
  bool dirty = false;
  for (int i = 0; i < b->n; i++) {
    gid_ctx* c = b->ctx[i];
    int rows = 0;
    bool found = false;
    for (auto& r : cache)
      if (r[0] == c->H && r[1] == c->W && r[2] == c->K) {
        rows = r[3];
        found = true;
      }
    if (!found) {
      float us[GID_AUTOTUNE_TIMINGS];
      if (int rc = gid_autotune(c, reps, &rows, us)) return bfail(b, rc, gid_last_error(c));
      if (rows <= 0) {  // batches run multi-launch loops: keep the fastest of those
        const int cand[4] = {2, 4, 8, 17};
        int jb = 0;
        for (int j = 1; j < GID_AUTOTUNE_TIMINGS; j++)
          if ((j < 4 || j >= 6) && us[j] > 0.f && us[j] < us[jb]) jb = j;
        rows = jb < 4 ? cand[jb] : (jb == 10 ? 16 : (cand[jb - 6] | GID_PCG_FUSED));
      }
      // the videos of a batch run at once: no context holds an L2 set-aside for itself
      gid_set_l2_window(c, 0);
      cache.push_back({c->H, c->W, c->K, rows});
      dirty = true;
    }
    if (rows <= 0) rows = 17;  // a cache line naming a single-launch loop: batches run the multi-kernel PCG
    if (int rc = gid_set_apply_tile(c, rows)) return bfail(b, rc, gid_last_error(c));
  }
  if (dirty && cache_path) {
    FILE* f = fopen(cache_path, "w");
    if (!f) return bfail(b, GID_ERR_INVALID_ARG, std::string("cannot write ") + cache_path);
    for (auto& r : cache) fprintf(f, "%d %d %d %d\n", r[0], r[1], r[2], r[3]);
    fclose(f);
  }
  return GID_OK;
}

// ---------------------------------------------------------------- misclustering correction

extern "C" int gid_correct_region(int H, int W, int K, const gid_weights* w, const float* rgb_dev,
                                  const uint8_t* labels_dev, const float* b_init_host, const uint8_t* region_dev,
                                  int n_outer, int m_inner, void* stream, int* best_out, double* sparsity_out,
                                  uint8_t* labels_out_dev) {
  gid::NvtxRange nvtx_range("gid_correct_region");
  if (!rgb_dev || !labels_dev || !b_init_host || !region_dev || !best_out)
    return fail(nullptr, GID_ERR_INVALID_ARG, "NULL argument");
  if (K < 1 || K > GID_MAX_K || H < 1 || W < 1) return fail(nullptr, GID_ERR_INVALID_ARG, "bad H, W or K");
  if (n_outer < 1 || m_inner < 1) return fail(nullptr, GID_ERR_INVALID_ARG, "n_outer, m_inner >= 1");
  const long HW = (long)H * W;
  std::vector<int> Hs(K, H), Ws(K, W), Ks(K, K);
  gid_batch* bt = nullptr;
  if (int rc = gid_batch_create(K, Hs.data(), Ws.data(), Ks.data(), w, 0, stream, &bt)) return rc;
  uint8_t* labs = nullptr;
  auto done = [&](int rc) {
    if (labs) cudaFree(labs);
    gid_batch_destroy(bt);
    return rc;
  };
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMalloc(&labs, (size_t)K * HW) != cudaSuccess) {
    cudaGetLastError();
    return done(fail(nullptr, GID_ERR_OOM, "candidate labels"));
  }
  // candidate k: the region's pixels labelled k (base colour k + 1)
  std::vector<const float*> rgbs(K, rgb_dev);
  std::vector<const uint8_t*> lp(K);
  for (int k = 0; k < K; k++) {
    k_relabel<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(labels_dev, region_dev, (uint8_t)k, labs + k * HW, HW);
    lp[k] = labs + k * HW;
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return done(fail(nullptr, GID_ERR_CUDA, "k_relabel", cudaGetErrorString(e)));
  for (int k = 0; k < K; k++)
    if (int rc = gid_set_base_colors(gid_batch_ctx(bt, k), b_init_host))
      return done(fail(nullptr, rc, "candidate base colours", gid_last_error(gid_batch_ctx(bt, k))));
  if (int rc = gid_batch_set_frames(bt, rgbs.data(), lp.data())) return done(fail(nullptr, rc, gid_batch_last_error(bt)));
  if (int rc = gid_batch_init(bt, 0)) return done(fail(nullptr, rc, gid_batch_last_error(bt)));
  if (int rc = gid_batch_run(bt, n_outer, m_inner)) return done(fail(nullptr, rc, gid_batch_last_error(bt)));
  int best = -1;
  double best_s = 0.0;
  for (int k = 0; k < K; k++) {
    double tot = 0.0, per[8];
    if (int rc = gid_energy_region(gid_batch_ctx(bt, k), region_dev, &tot, per))
      return done(fail(nullptr, rc, "candidate energy", gid_last_error(gid_batch_ctx(bt, k))));
    if (sparsity_out) sparsity_out[k] = per[5];
    if (best < 0 || per[5] < best_s) {
      best = k;
      best_s = per[5];
    }
  }
  *best_out = best;
  if (labels_out_dev) {
    k_relabel<<<(unsigned)((HW + 255) / 256), 256, 0, s>>>(labels_dev, region_dev, (uint8_t)best, labels_out_dev, HW);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fail(nullptr, GID_ERR_CUDA, "k_relabel", cudaGetErrorString(e)));
  }
  return done(GID_OK);
}
