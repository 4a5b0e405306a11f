"""Python binding of the C ABI in include/gid.h (argument marshalling only).

Every step of the solve runs in the CUDA library ``libgid.so`` built in-tree by
``paper_1908_01961_b300.build``; there is no Python or CPU fallback.  PyTorch is
used only for device memory (tensors whose ``data_ptr()`` is passed through) and
for the CUDA stream.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgid.so")

GID_OK = 0
PRECOND_JACOBI, PRECOND_BLOCK = 0, 1
RESIDENT = -1  # gid_set_apply_tile: the resident PCG loop (GID_PCG_RESIDENT)
FUSED = 256    # gid_set_apply_tile(rows | FUSED): one kernel per PCG step (GID_PCG_FUSED)
AUTOTUNE_LOOPS = (2, 4, 8, 17, 0, RESIDENT, 2 | FUSED, 4 | FUSED, 8 | FUSED, 17 | FUSED, 16)
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_STATE = -1, -2, -3, -4
ERR_TIMEOUT, ERR_NUMERIC = -5, -6
ENERGY_TERMS = ("data", "clustering", "r_sparsity", "r_consistency", "monochrome", "i_sparsity", "smoothness",
                "non_neg")
ERRORS = {-1: "GID_ERR_INVALID_ARG", -2: "GID_ERR_CUDA", -3: "GID_ERR_OOM", -4: "GID_ERR_STATE",
          -5: "GID_ERR_TIMEOUT", -6: "GID_ERR_NUMERIC"}
MAX_K = 10
MAX_PAIRS = 8
TERMS = ("data", "clustering", "r_sparsity", "r_consistency", "monochrome", "i_sparsity", "smoothness", "non_neg")
KINDS = ("frame", "init", "linearize", "apply", "update", "dense", "energy", "readout", "pcg")

# Every function include/gid.h declares.
EXPORTS = (
    "gid_default_weights", "gid_create", "gid_destroy", "gid_last_error", "gid_set_base_colors",
    "gid_get_base_colors", "gid_set_frame", "gid_init", "gid_run", "gid_get_layers", "gid_get_state",
    "gid_set_state", "gid_energy", "gid_solve_frame_host", "gid_stage_precompute", "gid_stage_linearize",
    "gid_stage_apply", "gid_stage_pcg", "gid_stage_dense_normal", "gid_launch_count", "gid_profile",
    "gid_profile_read", "gid_new_sequence", "gid_dense_refine_noalloc", "gid_set_apply_tile", "gid_get_pcg_layout",
    "gid_autotune", "gid_set_l2_window", "gid_get_l2_window",
    "gid_set_preconditioner", "gid_get_preconditioner", "gid_debug_inject", "gid_pcg_history",
    "gid_set_pcg_history",
    "gid_set_graphs", "gid_batch_create", "gid_batch_destroy", "gid_batch_last_error", "gid_batch_ctx",
    "gid_batch_set_frames", "gid_batch_init", "gid_batch_new_sequence", "gid_batch_run", "gid_batch_autotune",
    "gid_batch_set_worklist",
    "gid_net_create", "gid_net_destroy", "gid_net_last_error", "gid_net_num_params", "gid_net_launch_count",
    "gid_net_set_weights", "gid_net_get_weights", "gid_net_get_grads", "gid_net_forward", "gid_net_backward",
    "gid_net_adam_step", "gid_net_set_loss_weights", "gid_init_learned", "gid_base_color_step",
    "gid_solve_video_host", "gid_recombine", "gid_cluster", "gid_energy_region", "gid_correct_region",
)


class GidError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Weights(ctypes.Structure):
    _fields_ = [(n, ctypes.c_float) for n in (
        "lambda_data", "lambda_clustering", "lambda_rsparsity", "p", "lambda_rconsistency", "lambda_monochrome",
        "lambda_isparsity", "lambda_smoothness", "lambda_nonneg", "lambda_IR", "lambda_CR", "eps",
        "retinex_sharpness", "consistency_tau")] + [(n, ctypes.c_int) for n in (
            "nonneg_strict", "irls_half", "rcluster_follows_b", "temporal", "refine_base_colors",
            "n_spatial_pairs", "n_temporal_pairs")] + [
        ("spatial_offsets", ctypes.c_int * (2 * MAX_PAIRS)),
        ("temporal_offsets", ctypes.c_int * (2 * MAX_PAIRS)),
    ]


_lib = None


def load():
    """Load libgid.so (raises if it has not been built: no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_1908_01961_b300.build`")
    L = ctypes.CDLL(LIB_PATH)
    P, I, D, F = ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
    LL = ctypes.POINTER(ctypes.c_longlong)
    L.gid_default_weights.argtypes = [ctypes.POINTER(Weights)]
    L.gid_default_weights.restype = None
    L.gid_create.argtypes = [I, I, I, ctypes.POINTER(Weights), P, ctypes.POINTER(P)]
    L.gid_destroy.argtypes = [P]
    L.gid_destroy.restype = None
    L.gid_last_error.argtypes = [P]
    L.gid_last_error.restype = ctypes.c_char_p
    L.gid_set_base_colors.argtypes = [P, F]
    L.gid_get_base_colors.argtypes = [P, F]
    L.gid_set_frame.argtypes = [P, P, P]
    L.gid_init.argtypes = [P, I]
    L.gid_new_sequence.argtypes = [P]
    L.gid_run.argtypes = [P, I, I]
    L.gid_get_layers.argtypes = [P, P, P]
    L.gid_get_state.argtypes = [P, P]
    L.gid_set_state.argtypes = [P, P]
    L.gid_energy.argtypes = [P, D, D]
    L.gid_solve_frame_host.argtypes = [P, P, P, I, I, I, P, P, P]
    L.gid_stage_precompute.argtypes = [P, P, P, P]
    L.gid_stage_linearize.argtypes = [P, P, P]
    L.gid_stage_apply.argtypes = [P, P, P]
    L.gid_stage_pcg.argtypes = [P, I, P]
    L.gid_stage_dense_normal.argtypes = [P, D, D]
    L.gid_launch_count.argtypes = [P, LL]
    L.gid_profile.argtypes = [P, I]
    L.gid_profile_read.argtypes = [P, D, LL]
    L.gid_set_apply_tile.argtypes = [P, I]
    L.gid_get_pcg_layout.argtypes = [P] + [ctypes.POINTER(I)] * 4
    L.gid_set_preconditioner.argtypes = [P, I]
    L.gid_debug_inject.argtypes = [P, I, ctypes.c_longlong]
    L.gid_pcg_history.argtypes = [P, D, I, ctypes.POINTER(I)]
    L.gid_set_pcg_history.argtypes = [P, I]
    L.gid_get_preconditioner.argtypes = [P]
    L.gid_set_graphs.argtypes = [P, I]
    L.gid_autotune.argtypes = [P, I, ctypes.POINTER(ctypes.c_int), F]
    L.gid_dense_refine_noalloc.argtypes = [I, I, I, P, P, F, ctypes.POINTER(Weights), P, P, P, P,
                                           ctypes.c_char_p, I]
    L.gid_batch_create.argtypes = [I, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(Weights),
                                    I, P, ctypes.POINTER(P)]
    L.gid_batch_destroy.argtypes = [P]
    L.gid_batch_destroy.restype = None
    L.gid_batch_last_error.argtypes = [P]
    L.gid_batch_last_error.restype = ctypes.c_char_p
    L.gid_batch_ctx.argtypes = [P, I]
    L.gid_batch_ctx.restype = P
    L.gid_batch_set_frames.argtypes = [P, ctypes.POINTER(P), ctypes.POINTER(P)]
    L.gid_batch_init.argtypes = [P, I]
    L.gid_batch_new_sequence.argtypes = [P]
    L.gid_batch_run.argtypes = [P, I, I]
    L.gid_batch_autotune.argtypes = [P, ctypes.c_char_p, I]
    L.gid_set_l2_window.argtypes = [P, I]
    L.gid_get_l2_window.argtypes = [P]
    L.gid_batch_set_worklist.argtypes = [P, I]
    L.gid_net_create.argtypes = [I, ctypes.POINTER(I), ctypes.c_uint64, P, ctypes.POINTER(P)]
    L.gid_net_destroy.argtypes = [P]
    L.gid_net_destroy.restype = None
    L.gid_net_last_error.argtypes = [P]
    L.gid_net_last_error.restype = ctypes.c_char_p
    L.gid_net_num_params.argtypes = [P]
    L.gid_net_num_params.restype = ctypes.c_long
    L.gid_net_launch_count.argtypes = [P]
    L.gid_net_launch_count.restype = ctypes.c_longlong
    L.gid_net_set_weights.argtypes = [P, F]
    L.gid_net_get_weights.argtypes = [P, F]
    L.gid_net_get_grads.argtypes = [P, F]
    L.gid_net_forward.argtypes = [P, I, I, I, P, P, P, P, P]
    L.gid_net_backward.argtypes = [P, I, I, I, P, P, P, P, P, D]
    L.gid_net_adam_step.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.gid_net_set_loss_weights.argtypes = [P, ctypes.c_float, ctypes.c_float, ctypes.c_float]
    L.gid_init_learned.argtypes = [P, P, ctypes.c_float]
    L.gid_base_color_step.argtypes = [P]
    L.gid_solve_video_host.argtypes = [P, I, P, P, I, I, I, P, P, P]
    L.gid_recombine.argtypes = [P, F, F, P, P]
    L.gid_cluster.argtypes = [I, I, P, I, ctypes.c_float, P, P, F, ctypes.POINTER(I), ctypes.c_char_p, I]
    L.gid_energy_region.argtypes = [P, P, D, D]
    L.gid_correct_region.argtypes = [I, I, I, ctypes.POINTER(Weights), P, P, F, P, I, I, P, ctypes.POINTER(I), D, P]
    for n in EXPORTS:
        if n not in ("gid_default_weights", "gid_destroy", "gid_last_error", "gid_batch_destroy",
                     "gid_batch_last_error", "gid_batch_ctx", "gid_net_destroy", "gid_net_last_error",
                     "gid_net_num_params", "gid_net_launch_count"):
            getattr(L, n).restype = ctypes.c_int
    _lib = L
    return L


def default_weights(spatial_offsets=None, temporal_offsets=None, **overrides) -> Weights:
    """gid_default_weights() plus pair offsets ((n, 2) int arrays of (dy, dx)) and overrides."""
    w = Weights()
    load().gid_default_weights(ctypes.byref(w))
    if spatial_offsets is not None:
        so = np.asarray(spatial_offsets, np.int32).reshape(-1, 2)
        w.n_spatial_pairs = len(so)
        for i, v in enumerate(so.ravel()):
            w.spatial_offsets[i] = int(v)
    if temporal_offsets is not None:
        to = np.asarray(temporal_offsets, np.int32).reshape(-1, 2)
        w.n_temporal_pairs = len(to)
        for i, v in enumerate(to.ravel()):
            w.temporal_offsets[i] = int(v)
    for k, v in overrides.items():
        setattr(w, k, v)
    return w


def dense_refine_noalloc(X, rgb, b_init, weights=None, A=None, g=None, b=None, stream=None):
    """Base-colour step without any device allocation inside the library (see
    gid_dense_refine_noalloc in include/gid.h).  X: (K+4, H, W) and rgb: (3, H, W)
    float32 CUDA tensors; A (3, K, K) float64, g (3, K) float64 and b (K, 3)
    float32 are optional caller-allocated CUDA outputs."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())

    def check(t, name, dtype, shape):
        if t is None:
            return
        if not isinstance(t, torch.Tensor) or t.device != dev or t.dtype != dtype or tuple(t.shape) != shape \
                or not t.is_contiguous():
            raise ValueError(f"{name}: need a contiguous {dtype} tensor of shape {shape} on {dev}")

    if not isinstance(X, torch.Tensor) or X.dim() != 3:
        raise ValueError("X: need a (K+4, H, W) tensor")
    V, H, W = X.shape
    K = V - 4
    if not 1 <= K <= MAX_K:
        raise ValueError(f"X has {V} planes: K = {K} is outside 1..{MAX_K}")
    check(X, "X", torch.float32, (V, H, W))
    check(rgb, "rgb", torch.float32, (3, H, W))
    check(A, "A", torch.float64, (3, K, K))
    check(g, "g", torch.float64, (3, K))
    check(b, "b", torch.float32, (K, 3))
    bi = np.ascontiguousarray(b_init, dtype=np.float32).reshape(K, 3)
    w = weights if weights is not None else default_weights()
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    err = ctypes.create_string_buffer(256)
    rc = load().gid_dense_refine_noalloc(H, W, K, _ptr(X), _ptr(rgb), bi.ctypes.data_as(ctypes.POINTER(ctypes.c_float)),
                                         ctypes.byref(w), ctypes.c_void_p(s), _ptr(A), _ptr(g), _ptr(b), err, 256)
    if rc != GID_OK:
        raise GidError(rc, err.value.decode())
    return A, g, b


def cluster(rgb, k_max=10, merge_dist=0.2, labels=None, stream=None):
    """Chromaticity clustering of a (3, H, W) float32 CUDA frame (gid_cluster).
    Returns (labels (H, W) uint8 CUDA tensor, b_init (K', 3) numpy float32)."""
    import torch
    _, H, W = rgb.shape
    assert rgb.is_cuda and rgb.is_contiguous() and rgb.dtype == torch.float32
    labels = torch.empty((H, W), dtype=torch.uint8, device=rgb.device) if labels is None else labels
    b = np.zeros((MAX_K, 3), np.float32)
    k = ctypes.c_int()
    err = ctypes.create_string_buffer(256)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = load().gid_cluster(H, W, _ptr(rgb), k_max, merge_dist, ctypes.c_void_p(s), _ptr(labels),
                            b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(k), err, 256)
    if rc != GID_OK:
        raise GidError(rc, err.value.decode())
    return labels, b[:k.value].copy()


def correct_region(rgb, labels, b_init, region, weights=None, n_outer=8, m_inner=20, stream=None):
    """Misclustering correction of a region (gid_correct_region): rgb (3, H, W)
    float32, labels and region (H, W) uint8 CUDA tensors, b_init (K, 3).
    Returns (winning label, i-sparsity per candidate (K,), corrected labels)."""
    import torch
    _, H, W = rgb.shape
    b = np.ascontiguousarray(b_init, np.float32)
    K = b.shape[0]
    w = weights if weights is not None else default_weights()
    best = ctypes.c_int()
    sp = np.zeros(K)
    out = torch.empty((H, W), dtype=torch.uint8, device=rgb.device)
    s = stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream
    L = load()
    rc = L.gid_correct_region(H, W, K, ctypes.byref(w), _ptr(rgb), _ptr(labels),
                              b.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), _ptr(region), n_outer, m_inner,
                              ctypes.c_void_p(s), ctypes.byref(best), sp.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                              _ptr(out))
    if rc != GID_OK:
        raise GidError(rc, L.gid_last_error(None).decode())
    return best.value, sp, out


def _ptr(t):
    if t is None:
        return None
    return ctypes.c_void_p(t.data_ptr())


class Solver:
    """One gid_ctx: H x W frames, K base colours, on the current CUDA device."""

    def __init__(self, H: int, W: int, K: int, weights: Weights | None = None, stream=None):
        import torch
        self.torch = torch
        self.H, self.W, self.K, self.V = H, W, K, K + 4
        self.lib = load()
        self.weights = weights if weights is not None else default_weights()
        h = ctypes.c_void_p()
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        rc = self.lib.gid_create(H, W, K, ctypes.byref(self.weights), s, ctypes.byref(h))
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_last_error(None).decode())
        self.h = h

    def _chk(self, rc):
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, shape, dtype=None):
        t = self.torch
        return t.empty(shape, dtype=dtype or t.float32, device="cuda")

    def _check_dev(self, x, shape, dtype):
        t = self.torch
        assert isinstance(x, t.Tensor) and x.is_cuda and x.is_contiguous(), "need a contiguous CUDA tensor"
        assert tuple(x.shape) == tuple(shape) and x.dtype == dtype, (tuple(x.shape), shape, x.dtype, dtype)

    # -- colours
    def set_base_colors(self, b):
        b = np.ascontiguousarray(b, dtype=np.float32).reshape(self.K, 3)
        self._chk(self.lib.gid_set_base_colors(self.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def base_colors(self) -> np.ndarray:
        b = np.zeros((self.K, 3), np.float32)
        self._chk(self.lib.gid_get_base_colors(self.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return b

    # -- frame / state
    def set_frame(self, rgb, labels):
        self._check_dev(rgb, (3, self.H, self.W), self.torch.float32)
        self._check_dev(labels, (self.H, self.W), self.torch.uint8)
        self._chk(self.lib.gid_set_frame(self.h, _ptr(rgb), _ptr(labels)))

    def new_sequence(self):
        self._chk(self.lib.gid_new_sequence(self.h))

    def init(self, mode: int = 0):
        self._chk(self.lib.gid_init(self.h, mode))

    def init_learned(self, net: "Net", zero_below: float = 0.0):
        """Initial state from the warm-start network (gid_init_learned)."""
        self._chk(self.lib.gid_init_learned(self.h, net.h, zero_below))

    def run(self, n_outer: int, m_inner: int):
        self._chk(self.lib.gid_run(self.h, n_outer, m_inner))

    def set_graphs(self, enable: bool):
        self._chk(self.lib.gid_set_graphs(self.h, 1 if enable else 0))

    def layers(self, R=None, T=None):
        R = self._dev((3, self.H, self.W)) if R is None else R
        T = self._dev((self.K + 1, self.H, self.W)) if T is None else T
        self._chk(self.lib.gid_get_layers(self.h, _ptr(R), _ptr(T)))
        return R, T

    def recombine(self, b_new=None, gains=None, mask=None, out=None):
        """Edited image from the current layers (gid_recombine): new base colours
        (K, 3), per-layer gains (K,), a uint8 CUDA mask (H, W) of recoloured
        objects (j = colour index + 1).  Returns a (3, H, W) CUDA tensor."""
        F = ctypes.POINTER(ctypes.c_float)
        bn = None if b_new is None else np.ascontiguousarray(b_new, np.float32).reshape(self.K, 3)
        g = None if gains is None else np.ascontiguousarray(gains, np.float32).reshape(self.K)
        if mask is not None:
            self._check_dev(mask, (self.H, self.W), self.torch.uint8)
        out = self._dev((3, self.H, self.W)) if out is None else out
        self._chk(self.lib.gid_recombine(self.h, None if bn is None else bn.ctypes.data_as(F),
                                         None if g is None else g.ctypes.data_as(F), _ptr(mask), _ptr(out)))
        return out

    def state(self):
        X = self._dev((self.V, self.H, self.W))
        self._chk(self.lib.gid_get_state(self.h, _ptr(X)))
        return X

    def set_state(self, X):
        self._check_dev(X, (self.V, self.H, self.W), self.torch.float32)
        self._chk(self.lib.gid_set_state(self.h, _ptr(X)))

    def base_color_step(self):
        """One base-colour step on the current layers (gid_base_color_step)."""
        self._chk(self.lib.gid_base_color_step(self.h))

    def energy(self):
        tot = ctypes.c_double()
        per = (ctypes.c_double * 8)()
        self._chk(self.lib.gid_energy(self.h, ctypes.byref(tot), per))
        return tot.value, np.array(per[:])

    def energy_region(self, mask):
        """Energy terms evaluated at the pixels where the (H, W) uint8 CUDA mask is nonzero."""
        self._check_dev(mask, (self.H, self.W), self.torch.uint8)
        tot = ctypes.c_double()
        per = (ctypes.c_double * 8)()
        self._chk(self.lib.gid_energy_region(self.h, _ptr(mask), ctypes.byref(tot), per))
        return tot.value, np.array(per[:])

    def solve_frame_host(self, rgb, labels, init_mode, n_outer, m_inner, R=None, T=None, b=None):
        """Host-buffer entry point; rgb/labels/R/T/b are numpy (ideally pinned) arrays."""
        def p(a):
            return None if a is None else ctypes.c_void_p(a.ctypes.data)
        self._chk(self.lib.gid_solve_frame_host(self.h, p(rgb), p(labels), init_mode, n_outer, m_inner,
                                                p(R), p(T), p(b)))

    def solve_video_host(self, rgb, labels, first_init_mode, n_outer, m_inner, R=None, T=None, b=None):
        """Pipelined host-buffer entry point for a sequence (gid_solve_video_host);
        rgb (n, 3, H, W), labels (n, H, W) and the optional outputs are numpy
        arrays (ideally page-locked)."""
        def p(a):
            return None if a is None else ctypes.c_void_p(a.ctypes.data)
        self._chk(self.lib.gid_solve_video_host(self.h, rgb.shape[0], p(rgb), p(labels), first_init_mode, n_outer,
                                                m_inner, p(R), p(T), p(b)))

    # -- stages
    def stage_precompute(self):
        wsr = self._dev((self.H, self.W))
        ns, nt = self.weights.n_spatial_pairs, self.weights.n_temporal_pairs
        ws = self._dev((max(ns, 1), self.H, self.W))
        wt = self._dev((max(nt, 1), self.H, self.W))
        self._chk(self.lib.gid_stage_precompute(self.h, _ptr(wsr), _ptr(ws) if ns else None, _ptr(wt) if nt else None))
        return wsr, ws[:ns], wt[:nt]

    def stage_linearize(self):
        g, d = self._dev((self.V, self.H, self.W)), self._dev((self.V, self.H, self.W))
        self._chk(self.lib.gid_stage_linearize(self.h, _ptr(g), _ptr(d)))
        return g, d

    def stage_apply(self, p):
        self._check_dev(p, (self.V, self.H, self.W), self.torch.float32)
        q = self._dev((self.V, self.H, self.W))
        self._chk(self.lib.gid_stage_apply(self.h, _ptr(p), _ptr(q)))
        return q

    def stage_pcg(self, m_inner):
        d = self._dev((self.V, self.H, self.W))
        self._chk(self.lib.gid_stage_pcg(self.h, m_inner, _ptr(d)))
        return d

    def stage_dense_normal(self):
        A = np.zeros((3, self.K, self.K))
        g = np.zeros((3, self.K))
        D = ctypes.POINTER(ctypes.c_double)
        self._chk(self.lib.gid_stage_dense_normal(self.h, A.ctypes.data_as(D), g.ctypes.data_as(D)))
        return A, g

    # -- operator tile shape
    def set_apply_tile(self, rows: int):
        self._chk(self.lib.gid_set_apply_tile(self.h, rows))

    def pcg_history(self) -> np.ndarray:
        """rho_m = <r_m, z_m> of the latest Gauss-Newton step's PCG steps (gid_pcg_history)."""
        rho = np.zeros(64)
        n = ctypes.c_int()
        self._chk(self.lib.gid_pcg_history(self.h, rho.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 64,
                                           ctypes.byref(n)))
        return rho[:n.value].copy()

    def solve_logged(self, n_outer: int, m_inner: int, path=None):
        """gid_run one outer iteration at a time (PCG history recording on
        meanwhile), recording after each the exact energy per term, the PCG rho
        history of its Gauss-Newton step and the host wall time; returns the records and, with a path, appends them to
        it as JSON lines.  The state it reaches is the one gid_run(n_outer,
        m_inner) reaches when the base colours are refined every outer
        iteration or never (refine_base_colors 1 or 0)."""
        import json
        import time
        recs = []
        self._chk(self.lib.gid_set_pcg_history(self.h, 1))
        try:
            for n in range(n_outer):
                t0 = time.perf_counter()
                self.run(1, m_inner)
                total, per = self.energy()
                rho = self.pcg_history()
                recs.append({"outer": n + 1, "energy": total, "terms": dict(zip(ENERGY_TERMS, map(float, per))),
                             "pcg_rho": rho.tolist(), "pcg_steps": m_inner,
                             "wall_ms": 1000.0 * (time.perf_counter() - t0)})
        finally:
            self._chk(self.lib.gid_set_pcg_history(self.h, 0))
        if path is not None:
            with open(path, "a") as f:
                for r in recs:
                    f.write(json.dumps(r) + "\n")
        return recs

    def debug_inject(self, phantom_blocks: int = 0, spin_limit: int = 0):
        """Fault injection for tests (gid_debug_inject): grid-barrier participants
        that never arrive and the barrier's poll limit; (0, 0) restores the defaults."""
        self._chk(self.lib.gid_debug_inject(self.h, phantom_blocks, spin_limit))

    def run_checked(self, n_outer: int, m_inner: int):
        """gid_run, then the exact energy; if the solve failed numerically
        (GID_ERR_NUMERIC: non-finite energy or a singular base-colour system) or
        a device wait gave up (GID_ERR_TIMEOUT), the layers are rolled back to
        the state before the call (a copy kept here) and the error is raised.
        The base colours need no copy: a base-colour step whose system is not
        positive definite (NaN included) leaves them unchanged.  Returns the
        energy (total, per term)."""
        X0 = self.state().clone()
        try:
            self.run(n_outer, m_inner)
            return self.energy()
        except GidError as e:
            if e.code not in (ERR_NUMERIC, ERR_TIMEOUT):
                raise
            self.set_state(X0)
            raise

    def set_preconditioner(self, kind: str):
        """'jacobi' (default) or 'block' (per-pixel diagonal blocks of J^T J)."""
        k = {"jacobi": PRECOND_JACOBI, "block": PRECOND_BLOCK}[kind]
        self._chk(self.lib.gid_set_preconditioner(self.h, k))

    def preconditioner(self) -> str:
        return ("jacobi", "block")[self.lib.gid_get_preconditioner(self.h)]

    def autotune(self, reps: int = 10):
        """Pick the fastest PCG execution (tile rows, 0 = persistent, -1 = resident, rows | FUSED)
        on the current frame; returns (rows, {rows: us per PCG step})."""
        rows = ctypes.c_int()
        us = (ctypes.c_float * len(AUTOTUNE_LOOPS))()
        self._chk(self.lib.gid_autotune(self.h, reps, ctypes.byref(rows), us))
        return rows.value, dict(zip(AUTOTUNE_LOOPS, us[:]))

    def set_l2_window(self, on: bool):
        """Mark the operator coefficients persisting in L2 for the PCG launches (gid_set_l2_window)."""
        self._chk(self.lib.gid_set_l2_window(self.h, 1 if on else 0))

    def l2_window(self) -> bool:
        return self.lib.gid_get_l2_window(self.h) == 1

    def pcg_layout(self):
        """(rows of the current PCG loop, (tile_w, tile_h, blocks) of the resident loop on this
        frame, zeros if it does not fit) -- gid_get_pcg_layout."""
        v = [ctypes.c_int() for _ in range(4)]
        self._chk(self.lib.gid_get_pcg_layout(self.h, *[ctypes.byref(x) for x in v]))
        return v[0].value, (v[1].value, v[2].value, v[3].value)

    # -- instrumentation
    def launch_count(self) -> int:
        n = ctypes.c_longlong()
        self._chk(self.lib.gid_launch_count(self.h, ctypes.byref(n)))
        return n.value

    def profile(self, enable: bool):
        self._chk(self.lib.gid_profile(self.h, 1 if enable else 0))

    def profile_read(self):
        """{kind: (total ms, launches)} since the previous read."""
        ms = (ctypes.c_double * len(KINDS))()
        n = (ctypes.c_longlong * len(KINDS))()
        self._chk(self.lib.gid_profile_read(self.h, ms, n))
        return {k: (ms[i], n[i]) for i, k in enumerate(KINDS)}


class _BatchMember(Solver):
    """View of one video's context inside a Batch (owned by the batch)."""

    def __init__(self, handle, H, W, K, weights):
        import torch
        self.torch = torch
        self.H, self.W, self.K, self.V = H, W, K, K + 4
        self.lib = load()
        self.weights = weights
        self.h = ctypes.c_void_p(handle)

    def close(self):
        self.h = None  # the batch owns the context

    # A member context runs on its video's own stream: calls that exchange
    # device tensors with torch synchronise the device around the call.
    def _synced(name):
        def call(self, *a, **k):
            self.torch.cuda.synchronize()
            out = getattr(Solver, name)(self, *a, **k)
            self.torch.cuda.synchronize()
            return out
        call.__name__ = name
        return call

    state = _synced("state")
    set_state = _synced("set_state")
    layers = _synced("layers")
    set_frame = _synced("set_frame")
    stage_precompute = _synced("stage_precompute")
    stage_linearize = _synced("stage_linearize")
    stage_apply = _synced("stage_apply")
    stage_pcg = _synced("stage_pcg")
    del _synced


class Batch:
    """n videos of uneven size solved together: one CUDA graph launch per gid_batch_run."""

    def __init__(self, shapes, weights=None, stream=None):
        """shapes: list of (H, W, K); weights: one Weights or a list of n."""
        import torch
        self.lib = load()
        n = len(shapes)
        self.shapes = [tuple(s) for s in shapes]
        Hs = (ctypes.c_int * n)(*[s[0] for s in shapes])
        Ws = (ctypes.c_int * n)(*[s[1] for s in shapes])
        Ks = (ctypes.c_int * n)(*[s[2] for s in shapes])
        per_video = isinstance(weights, (list, tuple))
        if per_video:
            warr = (Weights * n)(*weights)
            wp = ctypes.cast(warr, ctypes.POINTER(Weights))
            self._w = warr
        else:
            self._w = weights if weights is not None else default_weights()
            wp = ctypes.pointer(self._w)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        h = ctypes.c_void_p()
        rc = self.lib.gid_batch_create(n, Hs, Ws, Ks, wp, 1 if per_video else 0, s, ctypes.byref(h))
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_batch_last_error(None).decode())
        self.h = h
        self.videos = [_BatchMember(self.lib.gid_batch_ctx(h, i), *self.shapes[i],
                                    warr[i] if per_video else self._w) for i in range(n)]

    def _chk(self, rc):
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_batch_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.videos = []
            self.lib.gid_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_frames(self, rgbs, labels):
        n = len(self.shapes)
        r = (ctypes.c_void_p * n)(*[t.data_ptr() for t in rgbs])
        l = (ctypes.c_void_p * n)(*[t.data_ptr() for t in labels])
        self._chk(self.lib.gid_batch_set_frames(self.h, r, l))

    def init(self, mode=0):
        self._chk(self.lib.gid_batch_init(self.h, mode))

    def new_sequence(self):
        self._chk(self.lib.gid_batch_new_sequence(self.h))

    def run(self, n_outer, m_inner):
        self._chk(self.lib.gid_batch_run(self.h, n_outer, m_inner))

    def autotune(self, cache_path=None, reps=5):
        self._chk(self.lib.gid_batch_autotune(self.h, cache_path.encode() if cache_path else None, reps))

    def set_worklist(self, on: bool, persistent: bool = False):
        """True: PCG steps as work-list launches over all videos of one K (default), or with
        persistent=True as one cooperative launch per K and Gauss-Newton step; False: one graph
        branch per video."""
        self._chk(self.lib.gid_batch_set_worklist(self.h, (2 if persistent else 1) if on else 0))


class Net:
    """One gid_net: the warm-start encoder-decoder for K base colours (include/gid.h)."""

    def __init__(self, K: int, widths=(32, 64, 96, 128), seed: int = 0, stream=None):
        import torch
        self.torch = torch
        self.K = K
        self.widths = tuple(int(w) for w in widths)
        self.lib = load()
        wd = (ctypes.c_int * 4)(*self.widths)
        s = ctypes.c_void_p(stream.cuda_stream if stream is not None else torch.cuda.current_stream().cuda_stream)
        h = ctypes.c_void_p()
        rc = self.lib.gid_net_create(K, wd, ctypes.c_uint64(seed), s, ctypes.byref(h))
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_net_last_error(None).decode())
        self.h = h
        self.n_params = int(self.lib.gid_net_num_params(h))

    def _chk(self, rc):
        if rc != GID_OK:
            raise GidError(rc, self.lib.gid_net_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.gid_net_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_weights(self, blob):
        b = np.ascontiguousarray(blob, dtype=np.float32).ravel()
        assert b.size == self.n_params, (b.size, self.n_params)
        self._chk(self.lib.gid_net_set_weights(self.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))

    def weights(self) -> np.ndarray:
        b = np.zeros(self.n_params, np.float32)
        self._chk(self.lib.gid_net_get_weights(self.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return b

    def grads(self) -> np.ndarray:
        b = np.zeros(self.n_params, np.float32)
        self._chk(self.lib.gid_net_get_grads(self.h, b.ctypes.data_as(ctypes.POINTER(ctypes.c_float))))
        return b

    def launch_count(self) -> int:
        return int(self.lib.gid_net_launch_count(self.h))

    def _inputs(self, rgb, labels, palette):
        t = self.torch
        B, C, H, W = rgb.shape
        for x, shape, dt in ((rgb, (B, 3, H, W), t.float32), (labels, (B, H, W), t.uint8),
                             (palette, (B, self.K, 3), t.float32)):
            assert x.is_cuda and x.is_contiguous() and tuple(x.shape) == shape and x.dtype == dt, (x.shape, shape)
        return B, H, W

    def forward(self, rgb, labels, palette, r=None, T=None):
        """rgb (B, 3, H, W), labels (B, H, W) uint8, palette (B, K, 3): CUDA tensors.
        Returns (r, T) = ((B, 3, H, W), (B, K+1, H, W)) float32 CUDA tensors."""
        t = self.torch
        B, H, W = self._inputs(rgb, labels, palette)
        r = t.empty((B, 3, H, W), device="cuda") if r is None else r
        T = t.empty((B, self.K + 1, H, W), device="cuda") if T is None else T
        self._chk(self.lib.gid_net_forward(self.h, B, H, W, _ptr(rgb), _ptr(labels), _ptr(palette), _ptr(r), _ptr(T)))
        return r, T

    def backward(self, rgb, labels, palette, r_target, T_target, sync_loss: bool = True):
        """Loss and weight gradients (kept in the network); returns the loss or None."""
        B, H, W = self._inputs(rgb, labels, palette)
        assert tuple(r_target.shape) == (B, 3, H, W) and tuple(T_target.shape) == (B, self.K + 1, H, W)
        assert r_target.is_contiguous() and T_target.is_contiguous()
        loss = ctypes.c_double()
        self._chk(self.lib.gid_net_backward(self.h, B, H, W, _ptr(rgb), _ptr(labels), _ptr(palette), _ptr(r_target),
                                            _ptr(T_target), ctypes.byref(loss) if sync_loss else None))
        return loss.value if sync_loss else None

    def set_loss_weights(self, w_r: float = 1.0, w_T0: float = 1.0, w_Tk: float = 1.0):
        self._chk(self.lib.gid_net_set_loss_weights(self.h, w_r, w_T0, w_Tk))

    def adam_step(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
        self._chk(self.lib.gid_net_adam_step(self.h, lr, beta1, beta2, eps))

    def train_step(self, rgb, labels, palette, r_target, T_target, lr, sync_loss=False):
        loss = self.backward(rgb, labels, palette, r_target, T_target, sync_loss)
        self.adam_step(lr)
        return loss
