"""The learned step on the largest mechanism (53 species, 325 reactions) with the
55 -> 2048 -> 1024 -> 512 -> 52 network, on the GPU against the oracle.

The same bounds as the 30-species tests (test_gpu_mlp.py, test_gpu_fp8.py), at
widths where the first layer's K (55, padded to 56 per BF16 term) leaves a
ragged k-block, the output layer is 52 wide, the epilogue runs its 64-species
instantiation and the bath closure covers 52 output species:
* forward (BF16): 99.99 % of outputs within 1e-2 (|u| + rms u) of the oracle
  with the device's BF16 rounding points, all within 3e-2;
* forward (E4M3 hidden-to-hidden layers): 99.9 % within 2e-2, all within 1e-1
  of the oracle's E4M3 emulation with the oracle's calibrated scales;
* chem_step_ann in both precisions: Y' within those bounds carried through dY
  and the renormalisation, sum Y' = 1, T' within 0.2 K (BF16) or 1 K (E4M3).
Several chunks and a ragged tail; weights, statistics and states are seeded.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu

HIDDEN = (2048, 1024, 512)


def _problem(n, seed):
    mech = synth.get_mech("c5")
    T, p, Y = synth.states_profiles(mech, n, seed, synth.padded_ld(n))
    widths = [mech.N + 2, *HIDDEN, mech.N - 1]
    layers = synth.mlp_layers(widths, 3000 + seed)
    x = M.features(T[:n], p[:n], Y[:, :n])
    mu_x, sd_x = M.zscore_stats(x)
    rng = np.random.default_rng(seed + 7)
    mu_u = rng.uniform(-1e-5, 1e-5, mech.N - 1)
    sd_u = 10.0 ** rng.uniform(-6, -3, mech.N - 1)
    stats = (mu_x, sd_x, mu_u, sd_u)
    z = np.asarray((x - mu_x) / sd_x, np.float32).astype(np.float64)
    scales = A.calibrate_fp8(layers, z)
    return mech, T, p, Y, widths, layers, stats, scales


def _net(widths, layers, stats, scales, chunk):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c5"), hidden=widths[1:4], chunk=chunk)
    assert net.widths == widths
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    binding.chem_mlp_set_fp8_scales(net, scales)
    return net


def _check_u(u, uq, frac_tol, all_tol, frac):
    rms = np.sqrt(np.mean(uq ** 2))
    err = np.abs(u - uq)
    assert np.mean(err <= frac_tol * (np.abs(uq) + rms)) >= frac, np.mean(err <= frac_tol * (np.abs(uq) + rms))
    bound = all_tol * (np.abs(uq) + rms)
    if not np.all(err <= bound):
        i, j = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d of %d outside; worst cell %d out %d: gpu %.6g oracle %.6g (rms %.3g)"
                             % ((err > bound).sum(), err.size, i, j, u[i, j], uq[i, j], rms))


TOL = {0: (1e-2, 3e-2, 0.9999, 0.2), 1: (2e-2, 1e-1, 0.999, 1.0)}   # prec -> frac_tol, all_tol, frac, T bound


@pytest.mark.parametrize("prec", [0, 1])
def test_c5_forward_parity(prec):
    import torch
    from paper_2312_05800_gb300 import binding
    n = 2600
    mech, T, p, Y, widths, layers, stats, scales = _problem(n, 2051)
    net = _net(widths, layers, stats, scales, chunk=1024)        # three chunks, the last ragged
    u = torch.full((n, 64), float("nan"), dtype=torch.float32, device="cuda")
    binding.chem_mlp_forward_prec(net, prec, n, T.shape[0], to_dev(T), to_dev(p), to_dev(Y), u, 64)
    torch.cuda.synchronize()
    assert net.error() == 0
    u = u.double().cpu().numpy()[:, :widths[4]]
    kw = {"round_bf16": True} if prec == 0 else {"fp8_scales": scales}
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], **kw)
    ft, at, fr, _ = TOL[prec]
    _check_u(u, uq, ft, at, fr)
    net.free()


@pytest.mark.parametrize("prec", [0, 1])
def test_c5_step_ann_parity(prec):
    import torch
    from paper_2312_05800_gb300 import binding
    n = 2600
    mech, T, p, Y, widths, layers, stats, scales = _problem(n, 2052)
    net = _net(widths, layers, stats, scales, chunk=1024)
    ld = T.shape[0]
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    binding.chem_step_ann(dev_mech("c5"), net, n, ld, 1e-6, prec, None, Td, pd, Yd, st)
    torch.cuda.synchronize()
    assert net.error() == 0
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    kw = {"round_bf16": True} if prec == 0 else {"fp8_scales": scales}
    To, Yo = A.step_ann(mech, layers, stats, T[:n], p[:n], Y[:, :n], **kw)
    assert np.all(st.cpu().numpy()[:n] == 0)
    assert np.abs(Yg[:, :n].sum(axis=0) - 1).max() < 1e-12 and Yg[:, :n].min() >= 0
    ft, at, fr, tb = TOL[prec]
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], **kw)
    bdy = (ft * (np.abs(uq) + np.sqrt(np.mean(uq ** 2))) * stats[3]).T
    sp = A.out_species(mech)
    btot = np.zeros_like(Yo)
    btot[sp, :] = bdy
    btot[mech.bath, :] = bdy.sum(axis=0)
    bound = btot + Yo * 2.0 * bdy.sum(axis=0)[None, :] + 1e-12
    err = np.abs(Yg[:, :n] - Yo)
    # the frac_tol bound holds for all but the rare rounding flips: allow the same fraction outside
    # it, and the all_tol bound (at / ft times wider) everywhere
    assert np.mean(err <= bound) >= fr, np.mean(err <= bound)
    wide = bound * (at / ft)
    if not np.all(err <= wide):
        k, i = np.unravel_index(np.argmax(err / wide), err.shape)
        raise AssertionError("%d outside; worst species %d cell %d: %.3g vs bound %.3g"
                             % ((err > wide).sum(), k, i, err[k, i], wide[k, i]))
    assert np.all(np.abs(Tg[:n] - To) <= tb + 1e-5 * To), np.abs(Tg[:n] - To).max()
    assert np.array_equal(Tg[n:], T[n:])
    net.free()
