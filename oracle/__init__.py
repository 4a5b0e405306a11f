"""FP64 CPU oracle for the illumination decomposition solve (test infrastructure).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline leg, never by the product library.  The
arithmetic lives in ``oracle.c`` (plain serial FP64 C); this module compiles it
with gcc, marshals numpy arrays through ctypes and adds the two steps the paper
runs outside the GPU solver: the small base-colour solve by SVD (Sec. 6.1) and
the outer flip-flop loop that alternates the Gauss-Newton step on the layers with
the base-colour step (Sec. 6.1, sparse-dense splitting).

Parity pins: see ``tests/test_oracle_*.py``.  The consistency prior of Sec. 5.1
is defined in the paper only by citation, so its reading here is "parity
unpinned" against the paper (only internal checks: finite-difference Jacobian,
symmetry, zero residual for constant r).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TERMS = ("data", "clustering", "r_sparsity", "r_consistency", "monochrome", "i_sparsity", "smoothness", "non_neg")
ALL = 0xFF

# Fixed parameter set of Sec. 7 ("Parameters"), eps of Sec. 5.3.1, sharpness 50 of Sec. 5.2.
DEFAULT_WEIGHTS = dict(
    lambda_data=5000.0, lambda_clustering=200.0, lambda_rsparsity=20.0, p=1.0,
    lambda_rconsistency=10.0, lambda_monochrome=10.0, lambda_isparsity=3.0,
    lambda_smoothness=3.0, lambda_nonneg=1000.0, lambda_IR=10.0, lambda_CR=100.0,
    eps=0.002, retinex_sharpness=50.0, tau=0.05, nonneg_strict=1, irls_half=0, rcluster_follows_b=0,
)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, -O2, strict IEEE: no -ffast-math;
    OpenMP spreads the loops over threads without changing any result)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        D = ctypes.POINTER(ctypes.c_double)
        P = ctypes.c_void_p
        _lib.or_apply.argtypes = [P, D, D, ctypes.c_uint, D, D]
        _lib.or_rhs.argtypes = [P, D, D, ctypes.c_uint, D]
        _lib.or_diag.argtypes = [P, D, D, ctypes.c_uint, D]
        _lib.or_surrogate.argtypes = [P, D, D, ctypes.c_uint, D]
        _lib.or_residuals.argtypes = [P, D, D, ctypes.c_uint, D, ctypes.POINTER(ctypes.c_int), ctypes.c_long]
        _lib.or_residuals.restype = ctypes.c_long
        _lib.or_energy.argtypes = [P, D, D]
        _lib.or_pcg.argtypes = [P, D, ctypes.c_int, D, D]
        _lib.or_gn_step.argtypes = [P, D, ctypes.c_int]
        _lib.or_block_diag.argtypes = [P, D, D, ctypes.c_uint, D]
        _lib.or_pcg_variant.argtypes = [P, D, ctypes.c_int, ctypes.c_int, ctypes.c_int, D, D]
        _lib.or_pcg_variant.restype = ctypes.c_int
        _lib.or_dense_normal.argtypes = [P, D, D, D]
        _lib.or_init_cold.argtypes = [P, D]
        _lib.or_set_threads.argtypes = [ctypes.c_int]
        _lib.or_max_threads.restype = ctypes.c_int
        _lib.or_precompute.argtypes = [ctypes.c_int, ctypes.c_int, D, D, ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                                       ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double,
                                       D, D, D, D]
    return _lib


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (the results do not depend on it)."""
    lib().or_set_threads(int(n))


def max_threads() -> int:
    return int(lib().or_max_threads())


class _Struct(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int), ("W", ctypes.c_int), ("K", ctypes.c_int)] + [
        (n, ctypes.c_double) for n in (
            "lambda_data", "lambda_clustering", "lambda_rsparsity", "p", "lambda_rconsistency",
            "lambda_monochrome", "lambda_isparsity", "lambda_smoothness", "lambda_nonneg",
            "lambda_IR", "lambda_CR", "eps")
    ] + [
        ("nonneg_strict", ctypes.c_int), ("irls_half", ctypes.c_int),
        ("n_spatial", ctypes.c_int), ("n_temporal", ctypes.c_int),
        ("off_spatial", ctypes.c_void_p), ("off_temporal", ctypes.c_void_p),
        ("I", ctypes.c_void_p), ("labels", ctypes.c_void_p), ("b", ctypes.c_void_p),
        ("wsr", ctypes.c_void_p), ("omega_s", ctypes.c_void_p), ("omega_t", ctypes.c_void_p),
        ("rprev", ctypes.c_void_p), ("b_init", ctypes.c_void_p), ("rcluster_follows_b", ctypes.c_int),
    ]


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def precompute(I, off_s, off_t=None, Iprev=None, tau=0.05, sharpness=50.0):
    """Per-frame inputs of the priors: C, w_SR, spatial and temporal pair weights."""
    I = _f64(I)
    _, H, W = I.shape
    off_s = np.ascontiguousarray(off_s, dtype=np.int32).reshape(-1, 2)
    off_t = np.zeros((0, 2), np.int32) if off_t is None else np.ascontiguousarray(off_t, dtype=np.int32).reshape(-1, 2)
    C = np.zeros((3, H, W))
    wsr = np.zeros((H, W))
    om_s = np.zeros((len(off_s), H, W))
    om_t = np.zeros((len(off_t), H, W))
    ip = _f64(Iprev) if Iprev is not None else None
    ci = ctypes.POINTER(ctypes.c_int)
    lib().or_precompute(H, W, _d(I), _d(ip) if ip is not None else None, len(off_s), off_s.ctypes.data_as(ci),
                        len(off_t), off_t.ctypes.data_as(ci), tau, sharpness, _d(C), _d(wsr), _d(om_s),
                        _d(om_t) if ip is not None else None)
    return C, wsr, om_s, (om_t if ip is not None else None)


class Problem:
    """One frame's decomposition problem; owns the arrays the C struct points to."""

    def __init__(self, I, labels, b_init, wsr, omega_s, off_s, omega_t=None, off_t=None, rprev=None, b=None,
                 **weights):
        """b_init: the clustered base colours (anchor of the refinement and of
        R_cluster); b: the current (refined) colours, default b_init."""
        w = dict(DEFAULT_WEIGHTS)
        w.update(weights)
        self.weights = w
        self.I = _f64(I)
        _, self.H, self.W = self.I.shape
        self.labels = np.ascontiguousarray(labels, dtype=np.uint8)
        self.b_init = _f64(b_init).copy()
        self.b = self.b_init.copy() if b is None else _f64(b).copy()
        self.K = self.b.shape[0]
        self.V = self.K + 4
        self.wsr = _f64(wsr)
        self.off_s = np.ascontiguousarray(off_s, dtype=np.int32).reshape(-1, 2)
        self.omega_s = _f64(omega_s)
        self.temporal = omega_t is not None and rprev is not None
        self.off_t = np.ascontiguousarray(off_t if off_t is not None else np.zeros((0, 2)), dtype=np.int32).reshape(-1, 2)
        self.omega_t = _f64(omega_t) if self.temporal else None
        self.rprev = _f64(rprev) if self.temporal else None
        s = _Struct()
        s.H, s.W, s.K = self.H, self.W, self.K
        for n in ("lambda_data", "lambda_clustering", "lambda_rsparsity", "p", "lambda_rconsistency",
                  "lambda_monochrome", "lambda_isparsity", "lambda_smoothness", "lambda_nonneg",
                  "lambda_IR", "lambda_CR", "eps"):
            setattr(s, n, float(w[n]))
        s.nonneg_strict, s.irls_half = int(w["nonneg_strict"]), int(w["irls_half"])
        s.n_spatial, s.n_temporal = len(self.off_s), (len(self.off_t) if self.temporal else 0)
        s.off_spatial, s.off_temporal = self.off_s.ctypes.data, self.off_t.ctypes.data
        s.I, s.labels, s.b = self.I.ctypes.data, self.labels.ctypes.data, self.b.ctypes.data
        s.wsr, s.omega_s = self.wsr.ctypes.data, self.omega_s.ctypes.data
        s.omega_t = self.omega_t.ctypes.data if self.temporal else None
        s.rprev = self.rprev.ctypes.data if self.temporal else None
        s.b_init = self.b_init.ctypes.data
        s.rcluster_follows_b = int(w["rcluster_follows_b"])
        self._s = s

    @property
    def ptr(self):
        return ctypes.byref(self._s)

    @property
    def shape(self):
        return (self.V, self.H, self.W)

    def set_b(self, b):
        self.b[...] = b

    def _x(self, X):
        X = _f64(X)
        assert X.shape == self.shape, (X.shape, self.shape)
        return X

    def init_cold(self):
        X = np.zeros(self.shape)
        lib().or_init_cold(self.ptr, _d(X))
        return X

    def energy(self, X):
        E = np.zeros(8)
        lib().or_energy(self.ptr, _d(self._x(X)), _d(E))
        return E

    def surrogate(self, X, Xw=None, mask=ALL):
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        E = np.zeros(8)
        lib().or_surrogate(self.ptr, _d(X), _d(Xw), mask, _d(E))
        return E

    def apply(self, X, p, Xw=None, mask=ALL):
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        p = self._x(p)
        q = np.zeros(self.shape)
        lib().or_apply(self.ptr, _d(X), _d(Xw), mask, _d(p), _d(q))
        return q

    def rhs(self, X, Xw=None, mask=ALL):
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        g = np.zeros(self.shape)
        lib().or_rhs(self.ptr, _d(X), _d(Xw), mask, _d(g))
        return g

    def diag(self, X, Xw=None, mask=ALL):
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        d = np.zeros(self.shape)
        lib().or_diag(self.ptr, _d(X), _d(Xw), mask, _d(d))
        return d

    def residuals(self, X, Xw=None, mask=ALL, with_terms=False):
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        n = lib().or_residuals(self.ptr, _d(X), _d(Xw), mask, None, None, 0)
        F = np.zeros(n)
        t = np.zeros(n, np.int32)
        lib().or_residuals(self.ptr, _d(X), _d(Xw), mask, _d(F), t.ctypes.data_as(ctypes.POINTER(ctypes.c_int)), n)
        return (F, t) if with_terms else F

    def pcg(self, X, M):
        X = self._x(X)
        delta = np.zeros(self.shape)
        rz = np.zeros(M + 1)
        lib().or_pcg(self.ptr, _d(X), int(M), _d(delta), _d(rz))
        return delta, rz

    def block_diag(self, X, Xw=None, mask=ALL):
        """Per-pixel (V, V) diagonal blocks of J^T J, shape (H, W, V, V)."""
        X = self._x(X)
        Xw = X if Xw is None else self._x(Xw)
        V = self.shape[0]
        B = np.zeros((self.shape[1], self.shape[2], V, V))
        lib().or_block_diag(self.ptr, _d(X), _d(Xw), mask, _d(B))
        return B

    def pcg_variant(self, X, M, block=False, single_reduction=False):
        """M PCG steps with the Jacobi or block-Jacobi preconditioner, in the
        textbook or the single-reduction recurrence (returns delta, rho history)."""
        X = self._x(X)
        delta = np.zeros(self.shape)
        rz = np.zeros(M + 1)
        if not lib().or_pcg_variant(self.ptr, _d(X), int(M), int(block), int(single_reduction), _d(delta), _d(rz)):
            raise ArithmeticError("a diagonal block is not positive definite")
        return delta, rz

    def gn_step(self, X, M):
        X = self._x(X).copy()
        lib().or_gn_step(self.ptr, _d(X), int(M))
        return X

    def dense_normal(self, X):
        A = np.zeros((3, self.K, self.K))
        g = np.zeros((3, self.K))
        lib().or_dense_normal(self.ptr, _d(self._x(X)), _d(A), _d(g))
        return A, g


def fit_direct(I, X, b):
    """T_0 that minimises the data term (eq:data-term) at each pixel with r,
    T_1..T_K and b fixed: the data residual is linear in T_0, so with
    R = exp(r) and A_c = sum_k b_kc T_k the minimiser is
    sum_c R_c (I_c - R_c A_c) / sum_c R_c^2, taken at 0 when negative (the
    layers are non-negative, eq:nonnegativityterm).  Returns the new X."""
    X = _f64(X).copy()
    I = _f64(I)
    b = _f64(b).reshape(-1, 3)
    R = np.exp(X[:3])
    A = np.einsum("kc,khw->chw", b, X[4:])
    X[3] = np.maximum(np.sum(R * (I - R * A), axis=0) / np.sum(R * R, axis=0), 0.0)
    return X


def recombine(X, b, b_new, gains, mask):
    """Layer recombination of Sec. 7.4 (recolouring, colour keying, spill
    suppression): out = R' * (T_0 + sum_k g_k b'_k T_k) with R'_c = R_c b'_jc /
    b_jc on the pixels whose mask is j in 1..K where b_jc != 0 (other pixels
    keep R).
    X (K+4, H, W), b and b_new (K, 3), gains (K,), mask (H, W) ints."""
    X = _f64(X)
    b, b_new, gains = _f64(b).reshape(-1, 3), _f64(b_new).reshape(-1, 3), _f64(gains).ravel()
    K = b.shape[0]
    R = np.exp(X[:3])
    S = X[3][None] + np.einsum("k,kc,khw->chw", gains, b_new, X[4:])
    ratio = np.ones((K + 1, 3))
    ratio[1:] = np.where(b != 0.0, b_new / np.where(b != 0.0, b, 1.0), 1.0)
    m = np.where(np.asarray(mask) <= K, np.asarray(mask), 0)
    return R * ratio[m].transpose(2, 0, 1) * S


def chromaticity(I):
    """C = I / (I_R + I_G + I_B + 1e-6) in FP64 (Sec. 4.1; the 1e-6 keeps black
    pixels finite)."""
    I = np.asarray(I, np.float64)
    s = (I[0] + I[1]) + I[2] + 1e-6
    return I / s[None]


CLUSTER_BINS = 10


def cluster(I, k_max, merge_dist=0.2, max_iter=100):
    """Chromaticity clustering of Sec. 4.1, steps in the paper's order:
    1. chromaticity C of every pixel (FP64);
    2. histogram with 10 partitions per axis of (C_R, C_G, C_B) in [0, 1]
       (values outside, from negative noisy channels, count in the edge bins);
    3. weighted k-means with the bins' mid-points as samples and their
       populations as weights, at most k_max clusters (initial centres: the
       k_max most populated bins, ties by bin index; iterate until no bin
       changes cluster, at most max_iter times);
    4. merging: while two centres are closer than merge_dist (Euclidean
       chromaticity distance), the smaller cluster (by population) joins the
       larger, whose centre becomes the population-weighted mean of both
       (closest pair first; empty clusters are dropped);
    5. every pixel is assigned to its closest centre (its own chromaticity,
       FP64 distances);
    6. initial base colours: the mean RGB of each cluster's pixels.
    Clusters are ordered by decreasing population (ties by centre order).
    Returns (labels (H, W) uint8, b_init (K', 3) float64, centres (K', 3))."""
    I = np.asarray(I)
    C = chromaticity(I)
    nb = CLUSTER_BINS
    idx = np.clip(np.floor(C * nb).astype(np.int64), 0, nb - 1)              # (3, H, W); outside [0, 1] -> edge bins
    flat = (idx[0] * nb + idx[1]) * nb + idx[2]
    hist = np.bincount(flat.ravel(), minlength=nb ** 3).astype(np.float64)
    mids = (np.stack(np.meshgrid(np.arange(nb), np.arange(nb), np.arange(nb), indexing="ij"), -1).reshape(-1, 3)
            + 0.5) / nb
    occ = np.nonzero(hist)[0]
    w, x = hist[occ], mids[occ]
    order = sorted(range(len(occ)), key=lambda i: (-w[i], occ[i]))
    k = min(k_max, len(occ))
    centres = x[order[:k]].copy()
    assign = np.full(len(occ), -1)
    for _ in range(max_iter):
        d = ((x[:, None, :] - centres[None, :, :]) ** 2).sum(-1)
        new = d.argmin(axis=1)
        if np.array_equal(new, assign):
            break
        assign = new
        for j in range(k):
            sel = assign == j
            if w[sel].sum() > 0:
                centres[j] = (w[sel][:, None] * x[sel]).sum(0) / w[sel].sum()
    pop = np.array([w[assign == j].sum() for j in range(k)])
    alive = [j for j in range(k) if pop[j] > 0]
    cen = {j: centres[j].copy() for j in alive}
    pw = {j: pop[j] for j in alive}
    while len(alive) > 1:
        best = None
        for a in range(len(alive)):
            for b in range(a + 1, len(alive)):
                ja, jb = alive[a], alive[b]
                dist = np.sqrt(((cen[ja] - cen[jb]) ** 2).sum())
                if dist < merge_dist and (best is None or dist < best[0]):
                    best = (dist, ja, jb)
        if best is None:
            break
        _, ja, jb = best
        big, small = (ja, jb) if (pw[ja], -ja) >= (pw[jb], -jb) else (jb, ja)
        cen[big] = (pw[big] * cen[big] + pw[small] * cen[small]) / (pw[big] + pw[small])
        pw[big] += pw[small]
        alive.remove(small)
    alive.sort(key=lambda j: (-pw[j], j))
    centres = np.array([cen[j] for j in alive])
    d = ((C[None] - centres[:, :, None, None]) ** 2).sum(1)                   # (K', H, W)
    labels = d.argmin(axis=0).astype(np.uint8)
    I64 = I.astype(np.float64)
    b = np.array([I64[:, labels == j].mean(axis=1) if np.any(labels == j) else centres[j]
                  for j in range(len(alive))])
    return labels, b, centres


def region_isparsity(X, region, lambda_isparsity=DEFAULT_WEIGHTS["lambda_isparsity"]):
    """The i-sparsity term (eq:shading-sparsity-term) summed over a region's pixels."""
    X = _f64(X)
    return lambda_isparsity * np.abs(X[4:])[:, np.asarray(region) != 0].sum()


def correct_region(I, labels, b_init, region, off_s, N, M):
    """Reflectance correction of a misclustered region (Sec. 4.2): for every
    candidate base colour, a full decomposition (cold start, N x M) with the
    region's pixels labelled with it; the candidate whose solution has the
    sparsest indirect illumination over the region (smallest i-sparsity term)
    wins.  Returns (winning label, i-sparsity per candidate)."""
    I = _f64(I)
    K = np.asarray(b_init).shape[0]
    C, wsr, om, _ = precompute(I, off_s)
    sp = []
    for k in range(K):
        lab = np.where(np.asarray(region) != 0, k, labels).astype(np.uint8)
        pb = Problem(I, lab, b_init, wsr, om, off_s)
        X, _, _ = solve_frame(pb, pb.init_cold(), N, M)
        sp.append(region_isparsity(X, region))
    sp = np.array(sp)
    return int(sp.argmin()), sp


def dense_solve(A, g):
    """Delta b (K, 3) from the three K x K blocks by SVD pseudo-inverse (Sec. 6.1)."""
    K = A.shape[1]
    db = np.zeros((K, 3))
    for c in range(3):
        U, s, Vt = np.linalg.svd(A[c])
        keep = s > s[0] * 1e-14
        db[:, c] = Vt[keep].T @ ((U[:, keep].T @ g[c]) / s[keep])
    return db


def solve_frame(pb: Problem, X, N: int, M: int, refine: bool = True, block: bool = False):
    """N outer flip-flop iterations (Sec. 6.1): a Gauss-Newton step on the layers
    (M PCG steps) with the base colours fixed, then the base-colour step with the
    layers fixed.  Returns the final X, b and the exact energy after each outer
    iteration (energy history has N + 1 rows, row 0 at the initial state).
    block: the PCG steps use the block-Jacobi preconditioner instead of Jacobi."""
    X = _f64(X).copy()
    hist = [pb.energy(X)]
    for _ in range(N):
        X = X + pb.pcg_variant(X, M, block=True)[0] if block else pb.gn_step(X, M)
        if refine:
            A, g = pb.dense_normal(X)
            pb.set_b(pb.b_init + dense_solve(A, g))
        hist.append(pb.energy(X))
    return X, pb.b.copy(), np.array(hist)
