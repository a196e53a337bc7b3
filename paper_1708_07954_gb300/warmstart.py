"""Learned warm start for the local solves: harvesting, GPU training, weights file.

The network (see include/dba.h, dba_mlp_*) is trained on the GPU by the
library's own kernels on targets harvested from long local solves of ADMM runs
on training scenes that share the benchmark workloads' geometry but not their
seeds (workload-2 geometry with seeds 2001-2004, workload-1 geometry with
seeds 2005-2008).  torch provides only the device buffers.

    python -m paper_1708_07954_gb300.warmstart        # trains and writes WEIGHTS
"""
from __future__ import annotations

import os
import time

import numpy as np

from . import build, dba
from . import scenes as S

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "warmstart.f32")
HARVEST_ITERS = (0, 1, 2, 4, 8, 16, 32, 64)


def training_scenes():
    out = [S.scene2(seed=2001 + k, n_pts=60000) for k in range(4)]
    out += [S.scene1(seed=2005 + k) for k in range(4)]
    return out


def harvest(scene, samples, target_steps=20, iters=HARVEST_ITERS, precision=dba.DBA_PREC_F32_LOCAL, stream=None):
    """Features and targets (torch CUDA tensors) at several ADMM iterations of one scene."""
    import torch

    per = max(1, samples // len(iters))
    stride = max(1, scene.n_obs // per)
    cap = (scene.n_obs + stride - 1) // stride
    feats, targs = [], []
    with dba.Solver(scene, precision=precision, stream=stream, ground_truth=False) as s:
        done = 0
        for k in iters:
            s.iterate(k - done, stats=False)
            done = k
            f = torch.empty((cap, dba.DBA_MLP_N_FEATURES), dtype=torch.float32, device="cuda")
            t = torch.empty((cap, dba.DBA_MLP_N_TARGETS), dtype=torch.float32, device="cuda")
            n = s.harvest(stride, target_steps, f.data_ptr(), t.data_ptr(), cap)
            feats.append(f[:n])
            targs.append(t[:n])
    return torch.cat(feats), torch.cat(targs)


def train(feats, targs, epochs=30, batch=4096, lr=2e-3, seed=0):
    mlp = dba.Mlp(seed)
    n = feats.shape[0]
    mlp.fit_normalizer(feats.data_ptr(), targs.data_ptr(), n)
    history = []
    for ep in range(epochs):
        rate = lr * (0.5 * (1 + np.cos(np.pi * ep / epochs)))  # cosine schedule
        history.append(mlp.train(feats.data_ptr(), targs.data_ptr(), n, 1, batch, float(rate), seed + ep))
    return mlp, history


def save(mlp, path=WEIGHTS):
    os.makedirs(os.path.dirname(path), exist_ok=True)
    mlp.get_params().astype("<f4").tofile(path)


def load(path=WEIGHTS):
    p = np.fromfile(path, dtype="<f4")
    if p.shape != (dba.DBA_MLP_N_PARAMS,):
        raise ValueError(f"{path}: expected {dba.DBA_MLP_N_PARAMS} float32 parameters")
    mlp = dba.Mlp(0)
    mlp.set_params(p)
    return mlp


def main():
    import torch

    build.build()
    dba.load()
    t0 = time.time()
    fs, ts = [], []
    for sc in training_scenes():
        f, t = harvest(sc, samples=300000)
        fs.append(f)
        ts.append(t)
    feats, targs = torch.cat(fs), torch.cat(ts)
    print(f"harvested {feats.shape[0]} local problems in {time.time() - t0:.1f} s", flush=True)
    t1 = time.time()
    mlp, hist = train(feats, targs)
    print(f"trained in {time.time() - t1:.1f} s; loss per epoch: " + " ".join(f"{h:.4f}" for h in hist), flush=True)
    save(mlp)
    print(f"wrote {WEIGHTS}")


if __name__ == "__main__":
    main()
