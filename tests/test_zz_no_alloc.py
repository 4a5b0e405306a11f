"""The allocation-free base-colour step against the context path and the oracle (GPU).

gid_dense_refine_noalloc serves callers that cannot allocate device memory
themselves -- code inside another framework's memory pool, real-time loops that
must not wait on the allocator, processes that are only handed device pointers.
It keeps its scratch in a static device array instead of a context.  This file
runs last so that a failure here cannot hide any other test's result; it must
pass alone in a fresh process and after every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from harness import Case

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def reference(case, X):
    """A, g and the refined colours from the existing context entry points."""
    s = case.solver()
    rgb, lab = case.gpu_inputs()
    s.set_frame(rgb, lab)
    s.set_state(X)
    A, g = s.stage_dense_normal()
    b = np.stack([case.b_init[:, c] + np.linalg.solve(A[c], g[c]) for c in range(3)], axis=1)
    return A, g, b, rgb


def state(case, seed):
    rng = np.random.default_rng(seed)
    X = np.zeros((case.K + 4, case.H, case.W))
    X[:3] = np.log(case.b_init[case.frames[0].labels]).transpose(2, 0, 1) + rng.normal(0, 0.1, (3, case.H, case.W))
    X[3] = rng.uniform(0.5, 1.2, (case.H, case.W))
    X[4:] = np.abs(rng.normal(0, 0.05, (case.K, case.H, case.W)))
    return torch.from_numpy(X.astype(np.float32)).cuda()


def test_noalloc_matches_context_path_twice_in_a_row():
    from paper_1908_01961_b300 import gid
    # two calls in a row on different problems: the second must not see the first's scratch
    for case, seed in ((Case(H=41, W=70, K=6, n_cells=9, seed=3), 1), (Case(H=48, W=64, K=4, n_cells=12, seed=5), 2)):
        X = state(case, seed)
        A_ref, g_ref, b_ref, rgb = reference(case, X)
        A = torch.zeros((3, case.K, case.K), dtype=torch.float64, device="cuda")
        g = torch.zeros((3, case.K), dtype=torch.float64, device="cuda")
        b = torch.zeros((case.K, 3), dtype=torch.float32, device="cuda")
        gid.dense_refine_noalloc(X, rgb, case.b_init, gid.default_weights(), A, g, b)
        A, g, b = A.cpu().numpy(), g.cpu().numpy(), b.cpu().numpy()
        assert np.abs(A - A_ref).max() <= 1e-5 * np.abs(A_ref).max()
        assert np.abs(g - g_ref).max() <= 1e-4 * np.abs(g_ref).max()
        assert np.abs(b - b_ref).max() <= 1e-5 * max(1.0, np.abs(b_ref).max())
        # and against the FP64 oracle's normal equations and SVD solve at the same (float32) layers
        pb = case.oracle_problem()
        A_o, g_o = pb.dense_normal(X.cpu().numpy().astype(np.float64))
        b_o = case.b_init + O.dense_solve(A_o, g_o)
        assert np.abs(A - A_o).max() <= 1e-5 * np.abs(A_o).max()
        assert np.abs(g - g_o).max() <= 1e-4 * np.abs(g_o).max()
        assert np.abs(b - b_o).max() <= 1e-4 * max(1.0, np.abs(b_o).max())


def test_noalloc_rejects_sizes_beyond_its_limit():
    from paper_1908_01961_b300 import gid
    lib = gid.load()
    err = ctypes.create_string_buffer(128)
    X = torch.zeros((15, 4, 4), device="cuda")
    rgb = torch.zeros((3, 4, 4), device="cuda")
    b0 = np.full((11, 3), 0.5, np.float32)
    w = gid.default_weights()
    rc = lib.gid_dense_refine_noalloc(4, 4, 11, ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(rgb.data_ptr()),
                                      b0.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), ctypes.byref(w), None,
                                      None, None, None, err, 128)
    assert rc == -1 and b"K must be" in err.value


def test_noalloc_binding_checks_its_tensors():
    """The binding refuses tensors the kernel would index wrongly (dtype, shape,
    layout, device) before calling into the library."""
    from paper_1908_01961_b300 import gid
    case = Case(H=16, W=24, K=3, n_cells=5, seed=4)
    X = state(case, 3)
    rgb, _ = case.gpu_inputs()
    ok = dict(A=torch.zeros((3, 3, 3), dtype=torch.float64, device="cuda"),
              g=torch.zeros((3, 3), dtype=torch.float64, device="cuda"),
              b=torch.zeros((3, 3), dtype=torch.float32, device="cuda"))
    bad = [dict(X=X.double()), dict(X=X.transpose(1, 2).contiguous().transpose(1, 2)), dict(X=X.cpu()),
           dict(rgb=rgb[:, :8]), dict(A=ok["A"].float()), dict(g=torch.zeros((3, 2), dtype=torch.float64,
                                                                              device="cuda")),
           dict(b=torch.zeros((2, 3), dtype=torch.float32, device="cuda"))]
    for change in bad:
        args = dict(X=X, rgb=rgb, **ok)
        args.update(change)
        with pytest.raises(ValueError):
            gid.dense_refine_noalloc(args["X"], args["rgb"], case.b_init, gid.default_weights(), args["A"],
                                     args["g"], args["b"])
    gid.dense_refine_noalloc(X, rgb, case.b_init, gid.default_weights(), **ok)
