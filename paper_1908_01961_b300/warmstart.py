"""Training and evaluation of the warm-start network (gid_net, include/gid.h).

The network learns to predict, from a frame and its clustered reflectance, the
decomposition that the plain solver reaches from its cold start (N = 8
Gauss-Newton steps of M = 20 PCG steps), so that a solve started from the
prediction needs fewer Gauss-Newton steps to reach the same energy.  The paper
has no network (Sec. 8 names learned priors as future work); everything here
runs through the library: the targets come from gid_run, the training from
gid_net_backward / gid_net_adam_step, the evaluation from gid_init_learned.

Data: seeded synthetic 640 x 480 frames with K = 6 (40 Voronoi cells, the
workload of the 30-frame video), each solved once; training samples are random
256 x 256 crops of those frames and of their solved layers.  Evaluation: held-
out frames (other seeds), each solved from the cold start and from the learned
start; the learned start's cost is the number of Gauss-Newton steps after
which its exact energy is at or below the cold start's final energy.

Command line:
    python -m paper_1908_01961_b300.warmstart train --frames 1000 --steps 6000 --out FILE.npy
    python -m paper_1908_01961_b300.warmstart evaluate --weights FILE.npy --eval-frames 20
    python -m paper_1908_01961_b300.warmstart sensitivity --eval-frames 4
    python -m paper_1908_01961_b300.warmstart finetune-energy --weights FILE.npy --frames 500 --steps 2000 \
        --lr 2e-4 --out FILE2.npy --eval-frames 50
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import time

import numpy as np

from . import gid, synth

H, W, K, N_CELLS, NOISE = 480, 640, 6, 40, 0.01
N_OUTER, M_INNER = 8, 20
TRAIN_SEED0, EVAL_SEED0 = 1_000_000, 2_000_000
WIDTHS = (32, 64, 96, 128)
# The indirect layers are small (a few hundredths) and sparse; without a larger
# factor their error hardly registers in the loss and the network predicts
# them as zero, a state the IRLS weights of Sec. 5.3 leave only slowly.
LOSS_WEIGHTS = (1.0, 1.0, 10.0)
# Predicted indirect values below this start at exactly zero (gid_init_learned).
# Swept over 0.002 .. 0.04 on held-out frames: below ~0.005 the first
# Gauss-Newton step overshoots small positive values below zero (non-negativity
# weight 0 for T > 0); above ~0.01 the start's indirect layers are mostly zero.
ZERO_BELOW = 0.01
HERE = os.path.dirname(os.path.abspath(__file__))
# the network trained on the plain solver's layers, then fine-tuned on the energy (train_energy)
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "warmstart_K6_energy.npy")


def solver_weights():
    """Solver settings of the single-frame solves: default term weights, the
    spatial pair offsets of seed 0, no temporal pairs."""
    off_s, _ = synth.offsets_for(0)
    return gid.default_weights(off_s)


def _make_frame(args):
    seed, t, noise = args
    v = synth.SyntheticVideo(H, W, K, N_CELLS, seed=seed, noise=noise)
    f = v.frame(t, noise=noise > 0)
    b = synth.initial_base_colors(f.I, f.labels, K)
    return f.I.astype(np.float32), f.labels.astype(np.uint8), b.astype(np.float32)


def generate(seeds, workers=None, noise=NOISE):
    """Frames (I, labels, b_init) for the given seeds; frame t = seed mod 30 of
    each seed's video (so the light direction varies as in the video)."""
    jobs = [(int(s), int(s) % 30, float(noise)) for s in seeds]
    workers = workers or max(1, min(32, (os.cpu_count() or 2) - 1, len(jobs)))
    if workers == 1:
        return [_make_frame(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_make_frame, jobs, chunksize=max(1, len(jobs) // (4 * workers)))


class Dataset:
    """Frames and their plain-solver layers, resident on the GPU."""

    def __init__(self, frames, n_outer=N_OUTER, m_inner=M_INNER, log=None):
        import torch
        n = len(frames)
        self.n = n
        self.rgb = torch.empty((n, 3, H, W), device="cuda")
        self.lab = torch.empty((n, H, W), dtype=torch.uint8, device="cuda")
        self.pal = torch.empty((n, K, 3), device="cuda")
        self.r = torch.empty((n, 3, H, W), device="cuda")
        self.T = torch.empty((n, K + 1, H, W), device="cuda")
        s = gid.Solver(H, W, K, solver_weights())
        t0 = time.time()
        for i, (I, lab, b) in enumerate(frames):
            self.rgb[i].copy_(torch.from_numpy(I))
            self.lab[i].copy_(torch.from_numpy(lab))
            self.pal[i].copy_(torch.from_numpy(b))
            s.set_base_colors(b)
            s.set_frame(self.rgb[i], self.lab[i])
            s.init(0)
            s.run(n_outer, m_inner)
            X = s.state()
            self.r[i].copy_(X[:3])
            self.T[i].copy_(X[3:])
            if log and (i + 1) % 200 == 0:
                log(f"solved {i + 1}/{n} frames ({time.time() - t0:.1f} s)")
        torch.cuda.synchronize()
        s.close()

    def crops(self, gen, batch, size):
        """A batch of random size x size crops (frame and offsets drawn from gen)."""
        import torch
        idx = torch.randint(self.n, (batch,), generator=gen).tolist()
        ys = torch.randint(0, (H - size) // 8 + 1, (batch,), generator=gen).mul(8).tolist()
        xs = torch.randint(0, (W - size) // 8 + 1, (batch,), generator=gen).mul(8).tolist()
        def cut(t, i, y, x):
            return t[i, ..., y:y + size, x:x + size]
        out = []
        for t in (self.rgb, self.lab, self.r, self.T):
            out.append(torch.stack([cut(t, i, y, x) for i, y, x in zip(idx, ys, xs)]).contiguous())
        pal = self.pal[idx].contiguous()
        return out[0], out[1], pal, out[2], out[3]


def train(net, data, steps, batch=8, size=256, lr=2e-3, lr_min=2e-5, seed=0, log=None, log_every=250):
    """Adam with a cosine learning-rate decay from lr to lr_min; returns the
    logged (step, loss) pairs."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    hist = []
    t0 = time.time()
    for step in range(steps):
        a = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(1, steps - 1)))
        rgb, lab, pal, r, T = data.crops(gen, batch, size)
        want = step % log_every == 0 or step == steps - 1
        loss = net.train_step(rgb, lab, pal, r, T, a, sync_loss=want)
        if want:
            hist.append((step, loss))
            if log:
                log(f"step {step} lr {a:.2e} loss {loss:.5f} ({time.time() - t0:.1f} s)")
    return hist


def train_energy(net, data, steps, batch=8, size=256, lr=2e-4, lr_min=2e-6, seed=0, m_inner=M_INNER, log=None,
                 log_every=250):
    """Fine-tuning on the decomposition energy (eq:giv-energy) itself: each step
    the network predicts the layers of a batch of crops, the solver takes one
    Gauss-Newton step of the energy from every prediction (the crop as a frame
    of its own: its pixels, labels and palette), and the network regresses onto
    the improved layers.  The gradient of the squared distance to them is, at
    the prediction, the Gauss-Newton descent direction of the energy, so the
    network is pulled toward states the solver would move to next, not toward
    a fixed plain-solver result.  Adam with a cosine learning-rate decay;
    returns the logged (step, loss, mean energy of the predictions) triples."""
    import torch
    gen = torch.Generator().manual_seed(seed)
    s = gid.Solver(size, size, K, solver_weights())
    hist = []
    t0 = time.time()
    for step in range(steps):
        a = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * step / max(1, steps - 1)))
        rgb, lab, pal, _, _ = data.crops(gen, batch, size)
        rp, Tp = net.forward(rgb, lab, pal)
        rt, Tt = torch.empty_like(rp), torch.empty_like(Tp)
        pal_h = pal.cpu().numpy()
        want = step % log_every == 0 or step == steps - 1
        e_sum = 0.0
        for i in range(batch):
            s.set_base_colors(pal_h[i])
            s.set_frame(rgb[i], lab[i])
            s.set_state(torch.cat([rp[i], Tp[i]]).contiguous())
            if want:
                e_sum += s.energy()[0]
            s.run(1, m_inner)
            X = s.state()
            rt[i].copy_(X[:3])
            Tt[i].copy_(X[3:])
        loss = net.train_step(rgb, lab, pal, rt, Tt, a, sync_loss=want)
        if want:
            hist.append((step, loss, e_sum / batch))
            if log:
                log(f"energy step {step} lr {a:.2e} loss {loss:.3e} mean crop energy {e_sum / batch:.4e} "
                    f"({time.time() - t0:.1f} s)")
    s.close()
    return hist


def energies(solver, n_outer=N_OUTER, m_inner=M_INNER):
    """Exact energy (total, and per term: rows of 8) after each of n_outer single
    Gauss-Newton steps; row 0 is the starting state."""
    tot, per = [], []
    for i in range(n_outer + 1):
        if i:
            solver.run(1, m_inner)
        t, p = solver.energy()
        tot.append(t)
        per.append(p)
    return np.array(tot), np.array(per)


def evaluate(net, frames, n_outer=N_OUTER, m_inner=M_INNER, zero_below=(None,), log=None, learned_steps=None):
    """Per frame: energies of the cold start after 0..n_outer Gauss-Newton
    steps and of the learned start after 0..learned_steps (default n_outer),
    and the learned start's step count to reach the cold start's final energy
    (learned_steps + 1 if it never does), for each threshold in zero_below
    (None = ZERO_BELOW)."""
    learned_steps = n_outer if learned_steps is None else learned_steps
    import torch
    s = gid.Solver(H, W, K, solver_weights())
    out = []
    for i, (I, lab, b) in enumerate(frames):
        rgb, lb = torch.from_numpy(I).cuda(), torch.from_numpy(lab).cuda()
        s.set_base_colors(b)
        s.set_frame(rgb, lb)
        s.init(0)
        Ec, Pc = energies(s, n_outer, m_inner)
        rec = dict(E_cold=Ec.tolist(), terms_cold=Pc.tolist(), learned={})
        for zb in zero_below:
            zb = ZERO_BELOW if zb is None else zb
            s.set_base_colors(b)
            s.init_learned(net, zb)
            El, Pl = energies(s, learned_steps, m_inner)
            hit = np.nonzero(El <= Ec[-1])[0]
            n_l = int(hit[0]) if len(hit) else learned_steps + 1
            rec["learned"][str(zb)] = dict(E=El.tolist(), terms=Pl.tolist(), n=n_l)
            if log:
                log(f"frame {i} zero_below {zb}: cold E {Ec[0]:.4e} -> {Ec[-1]:.4e}; learned E0 {El[0]:.4e}, "
                    f"reaches it after {n_l} steps")
        out.append(rec)
    s.close()
    return out


def sensitivity(frames, amplitudes=(0.001, 0.003, 0.01), blurs=(1.0, 2.0), seed=0, n_outer=N_OUTER,
                m_inner=M_INNER, log=None):
    """How accurate a start must be to save Gauss-Newton steps: per frame, the
    plain solve's result X* (cold start, n_outer steps) plus Gaussian noise of
    each amplitude (indirect values then clipped at 0), and X* blurred by a
    Gaussian of each width in pixels (the best a predictor of the solution's
    smooth part alone could do), each followed by one base-colour step, then
    the steps needed to return to the plain solve's final energy (n_outer + 1
    if not within n_outer)."""
    import torch
    from scipy.ndimage import gaussian_filter
    rng = np.random.default_rng(seed)
    s = gid.Solver(H, W, K, solver_weights())
    out = []
    for i, (I, lab, b) in enumerate(frames):
        rgb, lb = torch.from_numpy(I).cuda(), torch.from_numpy(lab).cuda()
        s.set_base_colors(b)
        s.set_frame(rgb, lb)
        s.init(0)
        s.run(n_outer, m_inner)
        E_star, _ = s.energy()
        Xs = s.state().cpu().numpy()
        rec = dict(E_star=E_star, steps={})
        starts = [(str(a), Xs + rng.normal(0.0, a, Xs.shape) if a else Xs.copy()) for a in (0.0,) + tuple(amplitudes)]
        starts += [(f"blur{sg}", np.stack([gaussian_filter(p, sg) for p in Xs])) for sg in blurs]
        for key, X0 in starts:
            X0[4:] = np.maximum(X0[4:], 0.0)
            s.set_base_colors(b)
            s.set_state(torch.from_numpy(np.ascontiguousarray(X0, np.float32)).cuda())
            s.base_color_step()
            E, _ = energies(s, n_outer, m_inner)
            hit = np.nonzero(E <= E_star)[0]
            rec["steps"][key] = int(hit[0]) if len(hit) else n_outer + 1
        out.append(rec)
        if log:
            log(f"frame {i}: steps back to the plain solve's energy by start noise RMS / blur width: {rec['steps']}")
    s.close()
    return out


def load_net(path=DEFAULT_WEIGHTS, stream=None):
    net = gid.Net(K, WIDTHS, stream=stream)
    net.set_weights(np.load(path))
    return net


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("cmd", choices=("train", "finetune-energy", "evaluate", "sensitivity"))
    ap.add_argument("--frames", type=int, default=1000)
    ap.add_argument("--steps", type=int, default=6000)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--loss-weights", type=float, nargs=3, default=LOSS_WEIGHTS, metavar=("W_R", "W_T0", "W_TK"))
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--weights", default=DEFAULT_WEIGHTS)
    ap.add_argument("--eval-frames", type=int, default=10)
    ap.add_argument("--eval-noise", type=float, default=NOISE, help="noise sigma of the evaluation frames")
    ap.add_argument("--zero-below", type=float, nargs="*", default=None,
                    help="thresholds of the learned start to evaluate (default: ZERO_BELOW)")
    ap.add_argument("--report", default=None, help="write a JSON summary here")
    a = ap.parse_args(argv)

    def log(m):
        print(m, flush=True)

    report = {}
    if a.cmd == "sensitivity":
        sens = sensitivity(generate(range(EVAL_SEED0, EVAL_SEED0 + a.eval_frames)), log=log)
        report.update(eval_frames=a.eval_frames, sensitivity=sens)
        if a.report:
            with open(a.report, "w") as f:
                json.dump(report, f, indent=1)
        return
    if a.cmd == "train":
        t0 = time.time()
        frames = generate(range(TRAIN_SEED0, TRAIN_SEED0 + a.frames))
        log(f"generated {len(frames)} frames in {time.time() - t0:.1f} s")
        t1 = time.time()
        data = Dataset(frames, log=log)
        del frames
        log(f"plain-solver targets in {time.time() - t1:.1f} s")
        net = gid.Net(K, WIDTHS, seed=a.seed)
        net.set_loss_weights(*a.loss_weights)
        t2 = time.time()
        hist = train(net, data, a.steps, a.batch, lr=a.lr, seed=a.seed, log=log)
        report.update(train_frames=a.frames, steps=a.steps, batch=a.batch, crop=256, lr=a.lr,
                      loss_weights=list(a.loss_weights),
                      train_seconds=time.time() - t2, loss=hist)
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        np.save(a.out, net.weights())
        log(f"saved {a.out}")
        del data
    elif a.cmd == "finetune-energy":
        net = load_net(a.weights)
        frames = generate(range(TRAIN_SEED0, TRAIN_SEED0 + a.frames))
        data = Dataset(frames, log=log)
        del frames
        t2 = time.time()
        hist = train_energy(net, data, a.steps, a.batch, lr=a.lr, seed=a.seed, log=log)
        report.update(start_weights=os.path.basename(a.weights), train_frames=a.frames, steps=a.steps,
                      batch=a.batch, crop=256, lr=a.lr, train_seconds=time.time() - t2, loss=hist)
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        np.save(a.out, net.weights())
        log(f"saved {a.out}")
        del data
    else:
        net = load_net(a.weights)
    if a.eval_frames > 0:
        zbs = a.zero_below or [ZERO_BELOW]
        ev = evaluate(net, generate(range(EVAL_SEED0, EVAL_SEED0 + a.eval_frames), noise=a.eval_noise),
                      zero_below=zbs, log=log)
        summary = {}
        for zb in zbs:
            n = [e["learned"][str(zb)]["n"] for e in ev]
            summary[str(zb)] = dict(n_learned=n, n_learned_max=max(n), mean_ratio=float(np.mean(n)) / N_OUTER)
            log(f"zero_below {zb}: learned start reaches the cold-start energy after {n} Gauss-Newton steps "
                f"(cold: {N_OUTER})")
        report.update(eval_frames=a.eval_frames, eval_noise=a.eval_noise, n_cold=N_OUTER, summary=summary, frames=ev)
    if a.report:
        with open(a.report, "w") as f:
            json.dump(report, f, indent=1)


if __name__ == "__main__":
    main()
