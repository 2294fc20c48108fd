"""chem_dense_bf16 (the tcgen05 GEMM behind every MLP layer, Sec. 3.2) against
an FP64 matrix product of the same BF16-rounded operands.

Bound: FP32 accumulation of exact BF16 products gives |err| <= 2^-22 K-scaled
sum |x||w| (we allow 1e-5 of that sum); a BF16 output adds 2^-8 relative.
Shapes cover every layer of both networks, ragged M, N and K, and every tile
width the library is built with."""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [  # (M, N, K)
    (300, 1600, 32), (1000, 800, 1600), (257, 400, 800), (4099, 29, 400),
    (129, 2048, 56), (131, 52, 512), (1, 16, 8), (640, 1024, 2048),
    # more tiles than CTAs: each persistent CTA reuses both TMEM accumulators
    (40000, 1600, 32), (20000, 800, 1600), (33333, 29, 400),
]


def _gelu64(z):
    from scipy.special import erf
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def _case(M, N, K, act, tile_n, seed):
    import torch
    from paper_2312_05800_gb300 import binding
    g = torch.Generator().manual_seed(seed)
    x = (torch.randn(M, K, generator=g) * 0.7).to(torch.bfloat16)
    W = (torch.randn(N, K, generator=g) / math.sqrt(K)).to(torch.bfloat16)
    b = torch.randn(N, generator=g, dtype=torch.float32) * 0.1
    xd, Wd, bd = x.cuda(), W.cuda(), b.cuda()
    err = torch.zeros(4, dtype=torch.int32, device="cuda")
    if act == 0:
        ldy = N + (-N) % 4
        y = torch.full((M, ldy), float("nan"), dtype=torch.float32, device="cuda")
    else:
        ldy = N + (-N) % 8
        y = torch.full((M, ldy), float("nan"), dtype=torch.bfloat16, device="cuda")
    binding.chem_dense_bf16(M, N, K, xd, K, Wd, K, bd, act, y, ldy, tile_n, err)
    torch.cuda.synchronize()
    assert int(err[0].item()) == 0
    x64, W64, b64 = x.double().numpy(), W.double().numpy(), b.double().numpy()
    acc = x64 @ W64.T + b64
    scale = np.abs(x64) @ np.abs(W64).T
    got = y.double().cpu().numpy()[:, :N]
    if act == 0:
        bound = 1e-5 * scale + 1e-6
        err = np.abs(got - acc)
    else:
        ref = _gelu64(acc)
        bound = 2.0 ** -8 * np.abs(ref) + 1.2e-5 * scale + 1e-6
        err = np.abs(got - ref)
    bad = err > bound
    if bad.any():
        i, j = np.unravel_index(np.argmax(err / bound), err.shape)
        raise AssertionError("%d of %d outside the bound; worst (%d, %d): err %.3g bound %.3g"
                             % (bad.sum(), bad.size, i, j, err[i, j], bound[i, j]))
    if ldy > N:   # padding columns untouched
        assert torch.isnan(y[:, N:].float()).all()


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("act", [0, 1])
def test_dense_auto_tile(M, N, K, act):
    _case(M, N, K, act, 0, 7 + M + N + K + act)


@pytest.mark.parametrize("tile_n", [32, 64, 128, 160, 208, 256])
def test_dense_every_tile_width(tile_n):
    _case(515, 450, 200, 1, tile_n, tile_n)
    _case(515, 450, 200, 0, tile_n, tile_n + 1)


def _bf16_round(a):
    a = np.ascontiguousarray(a, dtype=np.float32)
    b = a.view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("tile_n", [256, 208])
def test_gelu_epilogue_against_exact_gelu(tile_n):
    # The epilogue's GELU on exactly known pre-activations: X row m holds z_m in column 0, W row n
    # is the unit vector e_0, so the accumulator is z_m exactly and the epilogue sees
    # z = fl32(z_m + b_n). The device stores BF16(d) of its FP32 GELU value d. Every output g must
    # come from a d within the device GELU's error of the exact value (the erf polynomial's 8.0e-6
    # and FP32 rounding: delta = 4e-6 (1 + |z|)): the exact GELU lies within delta of the set of
    # FP32 values that round to g. Deep in the negative tail that set is near 0 and the test is
    # absolute, which is the accuracy the next layer sees.
    import torch
    from paper_2312_05800_gb300 import binding
    M, N, K = 8192, 512, 16
    rng = np.random.default_rng(31)
    zm = _bf16_round(np.concatenate([np.linspace(-12.0, 12.0, M - 2048), rng.normal(size=2048) * 2.0]))
    bn = (rng.uniform(-0.05, 0.05, N)).astype(np.float32)
    x = np.zeros((M, K), np.float32)
    x[:, 0] = zm
    W = np.zeros((N, K), np.float32)
    W[:, 0] = 1.0
    xd = torch.from_numpy(x).to(torch.bfloat16).cuda()
    Wd = torch.from_numpy(W).to(torch.bfloat16).cuda()
    bd = torch.from_numpy(bn).cuda()
    y = torch.empty((M, N), dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(4, dtype=torch.int32, device="cuda")
    binding.chem_dense_bf16(M, N, K, xd, K, Wd, K, bd, 1, y, N, tile_n, err)
    torch.cuda.synchronize()
    assert int(err[0].item()) == 0
    got = y.double().cpu().numpy()
    z = (zm[:, None].astype(np.float32) + bn[None, :]).astype(np.float64)   # fl32(z_m + b_n)
    exact = _gelu64(z)
    # half a BF16 unit in the last place of g (8 significant bits); 0 for g = 0
    _, ex = np.frexp(np.where(got != 0, np.abs(got), 1.0))
    hu = np.where(got != 0, np.ldexp(1.0, ex - 9), 0.0)
    dist = np.maximum(np.abs(exact - got) - hu, 0.0)
    delta = 4e-6 * (1.0 + np.abs(z))
    if not np.all(dist <= delta):
        i, j = np.unravel_index(np.argmax(dist / delta), dist.shape)
        raise AssertionError("%d of %d outside; worst z %.9g: device %.9g exact %.9g (delta %.3g)"
                             % ((dist > delta).sum(), dist.size, z[i, j], got[i, j], exact[i, j], delta[i, j]))
    # and the outputs are the correctly rounded ones almost everywhere the GELU is not tiny
    big = np.abs(exact) > 0.05
    assert np.mean(got[big] != _bf16_round(exact[big])) < 5e-3
