"""The reduced-precision (FP8-E4M3) forward on the GPU against the oracle.

* Weight quantisation: the E4M3 codes and per-row scales of both
  hidden-to-hidden layers equal the oracle's bit for bit (both sides divide in
  FP32 with correct rounding and round to nearest even).
* Calibration: the activation scales are max |h| / 448 of the BF16 forward; the
  device's maximum may sit one BF16 step from the oracle's, so 2^-7 relative.
* Forward: against the oracle's E4M3 emulation with the same scales. The two
  sides differ only where FP32 accumulation or the GELU's erf approximation
  (~4e-6) moves a value across an E4M3 or BF16 rounding boundary: 99.9 % of
  outputs within 2e-2 (|u| + rms u), all within 1e-1 (|u| + rms u).
* chem_step_ann at CHEM_PREC_FP8 carries that bound through dY and the
  renormalisation, like the BF16 test.
* Ragged widths (808, not a multiple of 16) take the element-store epilogue and
  a zero-filled K tail.
The scales passed to the device come from the oracle's calibration; no value
the oracle uses comes from the GPU.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M
from paper_2312_05800_gb300 import synth
from tests.gpu_util import dev_mech, to_dev

pytestmark = pytest.mark.gpu


def _problem(n, seed=2022, hidden=(1600, 800, 400)):
    mech = synth.get_mech("c2")
    T, p, Y = synth.states_profiles(mech, n, seed, synth.padded_ld(n))
    widths = [mech.N + 2, *hidden, mech.N - 1]
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


def _mlp(widths, layers, stats, **kw):
    from paper_2312_05800_gb300 import binding
    net = binding.Mlp(dev_mech("c2"), hidden=widths[1:4], **kw)
    net.set_params(synth.flatten_layers(layers))
    net.set_norm(*stats)
    return net


def _check_u(u, uq, frac_tol=2e-2, all_tol=1e-1, frac=0.999):
    rms = np.sqrt(np.mean(uq ** 2))
    err = np.abs(u - uq)
    assert np.mean(err <= frac_tol * (np.abs(uq) + rms)) >= frac, np.mean(err <= frac_tol * (np.abs(uq) + rms))
    bound = all_tol * (np.abs(uq) + rms)
    if not np.all(err <= bound):
        i, j = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d of %d outside; worst cell %d out %d: gpu %.6g oracle %.6g (rms %.3g)"
                             % ((err > bound).sum(), err.size, i, j, u[i, j], uq[i, j], rms))


def test_fp8_needs_scales_and_they_go_stale():
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats, scales = _problem(256)
    net = _mlp(widths, layers, stats)
    import torch
    u = torch.zeros((256, 32), dtype=torch.float32, device="cuda")
    args = (256, T.shape[0], to_dev(T), to_dev(p), to_dev(Y), u, 32)
    with pytest.raises(binding.ChemError):
        binding.chem_mlp_forward_prec(net, binding.CHEM_PREC_FP8, *args)
    binding.chem_mlp_set_fp8_scales(net, scales)
    binding.chem_mlp_forward_prec(net, binding.CHEM_PREC_FP8, *args)
    assert np.array_equal(binding.chem_mlp_get_fp8_scales(net), np.float32(scales))
    net.set_params(synth.flatten_layers(layers))      # new parameters: the E4M3 weights are stale
    with pytest.raises(binding.ChemError):
        binding.chem_mlp_forward_prec(net, binding.CHEM_PREC_FP8, *args)
    with pytest.raises(binding.ChemError):
        binding.chem_mlp_set_fp8_scales(net, [0.0, 1.0])
    net.free()


def test_fp8_weights_bit_exact():
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats, scales = _problem(64)
    W1 = np.array(layers[1][0])
    W1[5] = 0.0                                        # an all-zero row takes scale 1
    layers = [layers[0], (W1, layers[1][1]), layers[2], layers[3]]
    net = _mlp(widths, layers, stats)
    binding.chem_mlp_set_fp8_scales(net, scales)
    for l in (1, 2):
        codes, sw = binding.chem_mlp_get_fp8_weights(net, l)
        Wq, osw = A.quantize_rows(layers[l][0])
        assert np.array_equal(sw.astype(np.float64), osw)
        assert np.array_equal(A.e4m3_decode(codes), Wq)
    net.free()


def test_fp8_calibration_matches_oracle():
    from paper_2312_05800_gb300 import binding
    n = 5000
    mech, T, p, Y, widths, layers, stats, scales = _problem(n)
    net = _mlp(widths, layers, stats, chunk=2048)        # several chunks
    binding.chem_mlp_calibrate_fp8(net, n, T.shape[0], to_dev(T), to_dev(p), to_dev(Y))
    s = binding.chem_mlp_get_fp8_scales(net)
    assert np.allclose(s, scales, rtol=2.0 ** -7, atol=0)
    net.free()


@pytest.mark.parametrize("n,hidden", [(1000, (1600, 800, 400)), (20000, (1600, 800, 400)), (3001, (1600, 808, 400))])
def test_fp8_forward_parity(n, hidden):
    import torch
    from paper_2312_05800_gb300 import binding
    mech, T, p, Y, widths, layers, stats, scales = _problem(n, hidden=hidden)
    net = _mlp(widths, layers, stats, chunk=8192)       # several chunks and a ragged tail
    binding.chem_mlp_set_fp8_scales(net, scales)
    u = torch.full((n, 32), float("nan"), dtype=torch.float32, device="cuda")
    binding.chem_mlp_forward_prec(net, binding.CHEM_PREC_FP8, n, T.shape[0], to_dev(T), to_dev(p), to_dev(Y), u, 32)
    torch.cuda.synchronize()
    assert net.error() == 0
    u = u.double().cpu().numpy()[:, :widths[4]]
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], fp8_scales=scales)
    _check_u(u, uq)
    # and the reduced precision costs what E4M3 is expected to cost against FP64
    u64 = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n])
    assert np.sqrt(np.mean((u - u64) ** 2)) <= 0.25 * np.sqrt(np.mean(u64 ** 2))
    net.free()


def test_fp8_step_ann_parity():
    import torch
    from paper_2312_05800_gb300 import binding
    n = 3001
    mech, T, p, Y, widths, layers, stats, scales = _problem(n, seed=2032)
    net = _mlp(widths, layers, stats, chunk=1024)
    binding.chem_mlp_set_fp8_scales(net, scales)
    ld = T.shape[0]
    Td, pd, Yd = to_dev(T), to_dev(p), to_dev(Y)
    st = torch.full((ld,), -1, dtype=torch.int32, device="cuda")
    binding.chem_step_ann(dev_mech("c2"), net, n, ld, 1e-6, binding.CHEM_PREC_FP8, None, Td, pd, Yd, st)
    torch.cuda.synchronize()
    Tg, Yg = Td.cpu().numpy(), Yd.cpu().numpy()
    To, Yo = A.step_ann(mech, layers, stats, T[:n], p[:n], Y[:, :n], fp8_scales=scales)
    assert np.all(st.cpu().numpy()[:n] == 0)
    assert np.abs(Yg[:, :n].sum(axis=0) - 1).max() < 1e-12 and Yg[:, :n].min() >= 0
    sd_u = stats[3]
    uq = A.forward_u(mech, layers, stats, T[:n], p[:n], Y[:, :n], fp8_scales=scales)
    bdy = (1e-1 * (np.abs(uq) + np.sqrt(np.mean(uq ** 2))) * sd_u).T
    sp = A.out_species(mech)
    btot = np.zeros_like(Yo)
    btot[sp, :] = bdy
    btot[mech.bath, :] = bdy.sum(axis=0)
    bound = btot + Yo * 2.0 * bdy.sum(axis=0)[None, :] + 1e-12
    err = np.abs(Yg[:, :n] - Yo)
    if not np.all(err <= bound):
        k, i = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d outside; worst species %d cell %d: %.3g vs bound %.3g"
                             % ((err > bound).sum(), k, i, err[k, i], bound[k, i]))
    assert np.all(np.abs(Tg[:n] - To) <= 1.0 + 1e-5 * To), np.abs(Tg[:n] - To).max()
    assert np.array_equal(Tg[n:], T[n:])
    net.free()
