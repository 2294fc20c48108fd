"""Training-data generation and training loop of the learned chemistry.

Sec. 3.1: every sampled composition is integrated over dt = 1 us to give the
target; Sec. 3.2: the network is trained on (x, u*) pairs with Adam on the L1
loss (Eq. 5). Every numerical step runs in libchemgb.so (chem_step_stiff,
chem_mlp_fit_norm, mlp_train_step); this module only sequences the calls,
draws the seeded per-epoch permutation and holds the device buffers.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import binding, synth

DT = 1.0e-6
DATA_OPTS = dict(rtol=1e-4, atol_Y=1e-10, atol_T=1e-4, h0=1e-9, max_steps=20000)


@dataclass
class TrainingSet:
    """SoA pairs on the device: the state (T, p, Y) at t and (T1, Y1) at t + dt;
    the network's target is u* = Y1 - Y (computed inside the library)."""
    n: int
    ld: int
    T: object
    p: object
    Y: object
    Y1: object
    T1: object
    status: object


def make_training_set(mech: binding.Mech, smech: synth.Mech, n: int, seed: int, opts=None,
                      perturb_frac: float = 0.0) -> TrainingSet:
    """Samples n states (stratified premixed profiles; optionally a perturbed
    fraction), integrates them with the GPU stiff integrator over dt and keeps
    the pairs. Raises if any integration failed."""
    import torch
    ld = synth.padded_ld(n)
    T, p, Y = synth.states_profiles(smech, n, seed, ld)
    if perturb_frac > 0.0:
        T, Y, _ = synth.perturb_off_manifold(T, Y, n, perturb_frac, seed + 1)
    Td = torch.from_numpy(T).cuda()
    pd = torch.from_numpy(p).cuda()
    Yd = torch.from_numpy(Y).cuda()
    T1 = Td.clone()
    Y1 = Yd.clone()
    st = torch.zeros(ld, dtype=torch.int32, device="cuda")
    o = binding.make_opts(**(opts or DATA_OPTS))
    binding.chem_step_stiff(mech, n, ld, DT, o, T1, pd, Y1, st)
    nbad = int((st[:n] != 0).sum().item())
    if nbad:
        raise RuntimeError("%d training states failed to integrate" % nbad)
    return TrainingSet(n=n, ld=ld, T=Td, p=pd, Y=Yd, Y1=Y1, T1=T1, status=st)


def fit_norm(net: binding.Mlp, data: TrainingSet):
    binding.chem_mlp_fit_norm(net, data.n, data.ld, data.T, data.p, data.Y, data.Y1)


def train(net: binding.Mlp, data: TrainingSet, epochs: int, batch: int = 4096, lr0: float = 1e-3,
          lr_min: float = 1e-5, seed: int = 4003, log_every: int = 0, max_steps: int | None = None):
    """Adam with a cosine learning-rate schedule from lr0 to lr_min over the run;
    a seeded permutation of the training pairs per epoch. Returns the mean loss
    of each epoch (read back once per epoch)."""
    import torch
    rng = np.random.default_rng(seed)
    steps_per_epoch = max(1, data.n // batch)
    total = epochs * steps_per_epoch if max_steps is None else min(max_steps, epochs * steps_per_epoch)
    loss = torch.zeros(steps_per_epoch * 4, dtype=torch.float32, device="cuda")
    hist = []
    step = 0
    for ep in range(epochs):
        perm = torch.from_numpy(rng.permutation(data.n).astype(np.int32)).cuda()
        for b in range(steps_per_epoch):
            if step >= total:
                break
            lr = lr_min + 0.5 * (lr0 - lr_min) * (1.0 + math.cos(math.pi * step / max(1, total)))
            idx = perm[b * batch:(b + 1) * batch]
            binding.mlp_train_step(net, batch, idx, data.ld, data.T, data.p, data.Y, data.Y1, lr, loss[4 * b:])
            step += 1
        hist.append(float(loss[0:4 * steps_per_epoch:4].mean().item()))
        if log_every and (ep + 1) % log_every == 0:
            print("epoch %d loss %.5f" % (ep + 1, hist[-1]), flush=True)
        if step >= total:
            break
    return hist
