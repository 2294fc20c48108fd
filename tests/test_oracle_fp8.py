"""Pins of the oracle's reduced-precision (FP8-E4M3) forward.

* E4M3 rounding against torch's float8_e4m3fn conversion (a library routine:
  round to nearest even) for every value in range, including all midpoints
  between neighbouring E4M3 values; the 256 codes decoded from the format
  definition agree with torch's decoding; saturation at +-448 (the device's
  satfinite conversion) for larger values and infinities.
* Per-row weight quantisation: the largest |W| of a row lands on 448 exactly
  and every normal-range weight is reconstructed to within half an E4M3 step.
* The FP8 network on weights and activations that E4M3 represents exactly
  equals the BF16 network to FP32 rounding of the scales: this pins where the
  scales multiply and divide and which operand is transposed. On random
  weights it stays within the E4M3 error level of the FP64 network.
* The activation scales of the calibration, worked by hand for a network whose
  hidden activations are its biases' GELUs.
"""
import numpy as np
import pytest

from oracle import ann as A
from oracle import mlp as M


def test_e4m3_rounding_matches_torch_in_range():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = rng.standard_normal(200000) * np.exp(rng.uniform(-14, 6, 200000))
    x = x[np.abs(x) <= 448.0]
    codes = np.arange(256)
    v = A.e4m3_decode(codes)
    fin = np.unique(v[np.isfinite(v)])
    mids = (fin[:-1] + fin[1:]) / 2.0                     # exact ties: even mantissa wins
    x = np.concatenate([x, fin, mids, [0.0, -0.0, 2.0 ** -10, -2.0 ** -10, 3 * 2.0 ** -11]])
    x = x.astype(np.float32).astype(np.float64)
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(A.to_e4m3(x), ref)
    tdec = torch.from_numpy(codes.astype(np.uint8)).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(np.isnan(tdec), np.isnan(v))
    assert np.array_equal(tdec[np.isfinite(v)], v[np.isfinite(v)])


def test_e4m3_grid_from_the_format():
    v = A.e4m3_decode(np.arange(256))
    fin = v[np.isfinite(v)]
    assert fin.size == 254                                # two NaN codes, no infinities
    pos = np.unique(fin[fin > 0])
    assert pos.size == 126 and pos.max() == 448.0 and pos.min() == 2.0 ** -9
    assert 2.0 ** -6 in pos and 2.0 ** -6 - 2.0 ** -9 in pos  # smallest normal, largest subnormal
    assert np.array_equal(A.to_e4m3(fin), fin)            # every value is a fixed point
    # between neighbours the nearer one is chosen
    a, b = pos[:-1], pos[1:]
    assert np.array_equal(A.to_e4m3(a + 0.3 * (b - a)), a)
    assert np.array_equal(A.to_e4m3(a + 0.7 * (b - a)), b)


def test_e4m3_saturates():
    out = A.to_e4m3(np.array([448.0, 463.9, 464.0, 500.0, 1e30, np.inf, -1e9, -np.inf, np.nan]))
    assert np.array_equal(out[:8], [448, 448, 448, 448, 448, 448, -448, -448])
    assert np.isnan(out[8])


def test_quantize_rows():
    rng = np.random.default_rng(3)
    W = (rng.normal(size=(40, 300)) * 10.0 ** rng.uniform(-3, 1, (40, 1))).astype(np.float32).astype(np.float64)
    W[7] = 0.0
    W[3, :20] *= 1e-5                                      # E4M3 subnormals after scaling
    Wq, sw = A.quantize_rows(W)
    assert sw[7] == 1.0 and np.all(Wq[7] == 0)
    rows = [r for r in range(40) if r != 7]
    assert np.array_equal(np.abs(Wq[rows]).max(axis=1), np.full(39, 448.0))
    assert np.all(sw == sw.astype(np.float32))
    s = W[rows] / sw[rows, None]
    normal = np.abs(s) >= 2.0 ** -6
    rel = np.abs(Wq[rows] - s)[normal] / np.abs(s[normal])
    assert rel.max() <= 2.0 ** -4 * (1 + 1e-6)            # half a step of a 3-bit mantissa
    assert np.abs(Wq[rows] - s)[~normal].max() <= 2.0 ** -10 * (1 + 1e-6)


def _exact_layers():
    """Widths 6 -> 16 -> 16 -> 8 -> 3 with every E4M3 operand exactly representable:
    layer 1 has zero weights and biases in {12, ..., 28} (GELU is the identity there in
    FP64), the middle layers select one unit per row (a non-symmetric choice) or mix
    with weights in {+-1, +-1/2, +-1/4}."""
    rng = np.random.default_rng(11)
    W0 = np.zeros((16, 6))
    b0 = rng.choice([12.0, 16.0, 20.0, 24.0, 28.0], 16)
    perm = rng.permutation(16)
    W1 = np.zeros((16, 16))
    W1[np.arange(16), perm] = 1.0
    b1 = np.zeros(16)
    W2 = rng.choice([0.0, 1.0, -1.0, 0.5, -0.5, 0.25, -0.25], (8, 16))
    W2[:, 0] = 1.0                                         # every row's largest |w| is 1
    b2 = rng.normal(size=8)
    W3 = rng.normal(size=(3, 8)).astype(np.float32).astype(np.float64)
    b3 = rng.normal(size=3)
    return [(W0, b0), (W1, b1), (W2, b2), (W3, b3)]


def test_fp8_network_is_exact_on_representable_operands():
    layers = _exact_layers()
    z = np.random.default_rng(12).normal(size=(9, 6))
    s = (1.0 / 8.0, 1.0 / 8.0)            # h / s lands on E4M3 values 96 .. 224
    out8 = A.network(layers, z, fp8_scales=s)
    outb = A.network(layers, z, round_bf16=True)
    assert np.allclose(out8, outb, rtol=1e-6, atol=1e-9)
    # a transposed middle layer selects other units and is caught
    bad = list(layers)
    bad[1] = (layers[1][0].T.copy(), layers[1][1])
    assert not np.allclose(A.network(bad, z, fp8_scales=s), outb, rtol=1e-3, atol=1e-6)


def test_fp8_network_error_level_on_random_weights():
    layers = [(W, b) for W, b in
              ((L["W"], L["b"]) for L in M.init_params([10, 256, 128, 64, 6], seed=5))]
    z = np.random.default_rng(6).normal(size=(400, 10))
    s = A.calibrate_fp8(layers, z)
    h1 = A.to_bf16(M.gelu(A.split_bf16(z) @ A.to_bf16(layers[0][0]).T + layers[0][1]))
    assert np.isclose(np.abs(h1).max() / s[0], 448.0, rtol=1e-6)
    u8 = A.network(layers, z, fp8_scales=s)
    u64 = A.network(layers, z)
    # E4M3 keeps 3 mantissa bits (relative step 2^-3, rounding error <= 2^-4);
    # two quantised weight matrices and two quantised activations
    rel = np.sqrt(np.mean((u8 - u64) ** 2)) / np.sqrt(np.mean(u64 ** 2))
    assert 1e-4 < rel < 4 * 2.0 ** -4


def test_calibration_scales_worked_by_hand():
    # zero weights: the hidden activations are bf16(GELU(bias)) for every input row.
    # h1 = bf16(GELU(-9, 4, 2)) = (-0.0, 4.0, 1.953125): GELU(4) = 4 Phi(4) = 3.99987 rounds to 4,
    # GELU(2) = 1.9545 to the BF16 1.953125 and GELU(-9) is -1e-18; so s1 = fl32(4 / 448), where the
    # pre-activations' max |.| would have given 9 / 448.
    # h2 = bf16(GELU(1, -2, 8)) = (0.83984375, -0.0454..., 8.0): s2 = fl32(8 / 448).
    widths = [5, 3, 3, 2, 1]
    layers = [(np.zeros((o, i)), np.zeros(o)) for i, o in zip(widths[:-1], widths[1:])]
    layers[0] = (layers[0][0], np.array([-9.0, 4.0, 2.0]))
    layers[1] = (layers[1][0], np.array([1.0, -2.0, 8.0]))
    z = np.random.default_rng(3).normal(size=(7, 5))
    s = A.calibrate_fp8(layers, z)
    assert s == [float(np.float32(4.0 / 448.0)), float(np.float32(8.0 / 448.0))]
