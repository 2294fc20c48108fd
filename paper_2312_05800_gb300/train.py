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
                      perturb_frac: float = 0.0, hfrd: bool = False) -> TrainingSet:
    """Samples n states (stratified premixed profiles; optionally a perturbed
    fraction; or, with hfrd, the random states of Sec. 3.1 from hfrd_states, about
    n of them), integrates them with the GPU stiff integrator over dt and keeps
    the pairs. Raises if any integration failed."""
    import torch
    if hfrd:
        n, ld, Td, pd, Yd = hfrd_states(mech, smech, n, seed)
    else:
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


def lean_equilibrium(mech: binding.Mech, smech: synth.Mech, phi: float = 0.45, T0: float = 300.0,
                     p: float = synth.P_ATM, t_end: float = 1.0):
    """The lean-mixing endpoint of Sec. 3.1: the adiabatic, isobaric equilibrium of the fuel / air
    mixture at phi. Its complete-combustion products start at the temperature that keeps the
    unburnt mixture's enthalpy (Newton steps T -= (h - h0) / cp with props_eval in FP64), then the
    stiff integrator takes them to rest over t_end. Returns (T_eq, Y_eq) as host values."""
    import torch
    Yu, Yb = synth.fuel_air(smech, phi)
    N = smech.N
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
    Td = dev(np.full(4, T0))
    pd = dev(np.full(4, p))
    Yd = dev(np.repeat(Yu[:, None], 4, axis=1))
    cp = torch.zeros(4, dtype=torch.float64, device="cuda")
    h = torch.zeros_like(cp)
    binding.props_eval(mech, 1, 4, binding.CHEM_F64, Td, pd, Yd, cp, h)
    h0 = float(h[0].item())
    Yd.copy_(dev(np.repeat(Yb[:, None], 4, axis=1)))
    T = 2000.0
    for _ in range(100):
        Td.fill_(T)
        binding.props_eval(mech, 1, 4, binding.CHEM_F64, Td, pd, Yd, cp, h)
        d = (float(h[0].item()) - h0) / float(cp[0].item())
        T -= d
        if abs(d) < 1e-10:
            break
    Td.fill_(T)
    st = torch.zeros(4, dtype=torch.int32, device="cuda")
    o = binding.make_opts(rtol=1e-10, atol_Y=1e-16, atol_T=1e-10, h0=1e-9, max_steps=200000)
    binding.chem_step_stiff(mech, 1, 4, t_end, o, Td, pd, Yd, st)
    if int(st[0].item()) != 0:
        raise RuntimeError("equilibrium integration failed with status %d" % int(st[0].item()))
    return float(Td[0].item()), Yd[:N, 0].cpu().numpy()


def hfrd_states(mech: binding.Mech, smech: synth.Mech, n_base: int, seed: int, lean_frac: float = 0.1,
                t_min: float = 500.0):
    """Random training states of Sec. 3.1 on the GPU: base states (the profile sampler standing in
    for the flamelets) with T >= t_min perturbed by Eq. 1-4 with seeded uniform draws and filtered
    by Table 1 (chem_hfrd_perturb), plus lean_frac as many lean-mixing states blended between the
    phi = 0.45 adiabatic equilibrium and air (chem_hfrd_blend). Returns (n, ld, T, p, Y) on the
    device (SoA, ld a multiple of 4)."""
    import torch
    rng = np.random.default_rng(seed)
    ldb = synth.padded_ld(n_base)
    Tb, pb, Yb = synth.states_profiles(smech, n_base, seed, ldb)
    base = np.flatnonzero(Tb[:n_base] >= t_min)
    nb = base.size
    ld = synth.padded_ld(nb)
    T = np.zeros(ld); p = np.zeros(ld); Y = np.zeros((smech.N, ld))
    T[:nb], p[:nb], Y[:, :nb] = Tb[base], pb[base], Yb[:, base]
    b = smech.bath
    prm = binding.hfrd_params(T_min=T[:nb].min(), T_max=T[:nb].max(), p_min=p[:nb].min(), p_max=p[:nb].max(),
                              Yb_min=Y[b, :nb].min(), Yb_max=Y[b, :nb].max())
    c = np.zeros((3 + smech.N, ld))
    c[:, :nb] = rng.uniform(-1.0, 1.0, (3 + smech.N, nb))
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    T2 = torch.zeros(ld, dtype=torch.float64, device="cuda")
    p2 = torch.zeros_like(T2)
    Y2 = torch.zeros((smech.N, ld), dtype=torch.float64, device="cuda")
    keep = torch.zeros(ld, dtype=torch.uint8, device="cuda")
    binding.chem_hfrd_perturb(mech, prm, synth.element_table(smech), nb, ld, dev(T), dev(p), dev(Y), dev(c), T2, p2,
                              Y2, keep)
    kept = torch.nonzero(keep[:nb]).flatten()
    nk = int(kept.numel())
    nl = int(round(lean_frac * nk))
    n = nk + nl
    ldo = synth.padded_ld(n)
    To = torch.zeros(ldo, dtype=torch.float64, device="cuda")
    po = torch.full((ldo,), synth.P_ATM, dtype=torch.float64, device="cuda")
    Yo = torch.zeros((smech.N, ldo), dtype=torch.float64, device="cuda")
    To[:nk] = T2[kept]
    po[:nk] = p2[kept]
    Yo[:, :nk] = Y2[:, kept]
    if nl:
        Te, Ye = lean_equilibrium(mech, smech)
        s = dev(np.concatenate([rng.uniform(0.0, 1.0, nl), np.zeros(synth.padded_ld(nl) - nl)]))
        Tl = torch.zeros(synth.padded_ld(nl), dtype=torch.float64, device="cuda")
        Yl = torch.zeros((smech.N, synth.padded_ld(nl)), dtype=torch.float64, device="cuda")
        binding.chem_hfrd_blend(smech.N, nl, Tl.shape[0], s, Te, Ye, 300.0, synth.air(smech), Tl, Yl)
        To[nk:n] = Tl[:nl]
        Yo[:, nk:n] = Yl[:, :nl]
    return n, ldo, To, po, Yo


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


# ---------------------------------------------------------------------------
# data-parallel training: each rank a shard of every batch, one gradient all-reduce per step
# ---------------------------------------------------------------------------

def shard_rows(rows, rank: int, world: int):
    """Rank's contiguous, equal share of a batch's rows (len(rows) a multiple of world)."""
    n = len(rows) // world
    if n * world != len(rows):
        raise ValueError("the batch does not split into %d equal shards" % world)
    return rows[rank * n:(rank + 1) * n]


def allreduce_mean_(tensors, world: int, group=None):
    """Each tensor summed over the ranks, in place, then divided by world: with Eq. 5 averaged over
    each shard, the mean over equal shards is the gradient of the whole batch."""
    import torch.distributed as dist
    for t in tensors:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        t.div_(world)
    return tensors


def train_step_dp(net: binding.Mlp, rows, data: TrainingSet, lr: float, rank: int, world: int, loss=None,
                  group=None):
    """One data-parallel step: this rank's shard of the batch rows (int32, device) through
    mlp_train_grads, the mean of the handle's gradient buffers over the ranks (in place), then
    mlp_adam_step. Ranks that start with the same parameters and Adam state end with the same."""
    shard = shard_rows(rows, rank, world)
    binding.mlp_train_grads(net, len(shard), shard, data.ld, data.T, data.p, data.Y, data.Y1, loss)
    if world > 1:
        allreduce_mean_(binding.grad_buffers(net), world, group)
    binding.mlp_adam_step(net, lr)

