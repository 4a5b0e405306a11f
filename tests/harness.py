"""Shared test inputs: one seeded synthetic frame (or video) laid out for both
the oracle (float64 numpy) and the CUDA library (float32 torch tensors)."""
import numpy as np

import oracle as O
from paper_1908_01961_b300 import synth


class Case:
    def __init__(self, H, W, K, n_cells, seed=0, frames=1, temporal=False, noise=0.01):
        self.H, self.W, self.K = H, W, K
        self.video = synth.SyntheticVideo(H, W, K, n_cells, seed=seed, noise=noise)
        self.frames = [self.video.frame(t) for t in range(frames)]
        self.off_s, self.off_t = synth.offsets_for(seed)
        self.temporal = temporal
        f0 = self.frames[0]
        self.b_init = synth.initial_base_colors(f0.I, f0.labels, K).astype(np.float32).astype(np.float64)

    def oracle_problem(self, t=0, rprev=None, b=None, **w):
        """The oracle's problem for frame t, on the float32-rounded inputs the GPU sees."""
        f = self.frames[t]
        I = f.I.astype(np.float32).astype(np.float64)
        if self.temporal and t > 0 and rprev is not None:
            Ip = self.frames[t - 1].I.astype(np.float32).astype(np.float64)
            C, wsr, om_s, om_t = O.precompute(I, self.off_s, self.off_t, Iprev=Ip)
            return O.Problem(I, f.labels, self.b_init, wsr, om_s, self.off_s, omega_t=om_t, off_t=self.off_t,
                             rprev=rprev, b=b, **w)
        C, wsr, om_s, _ = O.precompute(I, self.off_s)
        return O.Problem(I, f.labels, self.b_init, wsr, om_s, self.off_s, b=b, **w)

    def gpu_inputs(self, t=0):
        import torch
        f = self.frames[t]
        rgb = torch.from_numpy(f.I.astype(np.float32)).cuda().contiguous()
        lab = torch.from_numpy(f.labels.astype(np.uint8)).cuda().contiguous()
        return rgb, lab

    def solver(self, **overrides):
        from paper_1908_01961_b300 import gid
        w = gid.default_weights(self.off_s, self.off_t if self.temporal else None,
                                temporal=1 if self.temporal else 0, **overrides)
        s = gid.Solver(self.H, self.W, self.K, w)
        s.set_base_colors(self.b_init)
        return s
