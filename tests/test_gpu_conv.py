"""The surrogate's tensor-core layers (include/mpw_surrogate.h) against the
numpy oracle (oracle/surrogate.py), element by element.

Both sides get the same bfloat16 operands; the oracle accumulates in FP64.
FP32 results must lie within 2e-5 of the sum of the absolute values of the
terms (sum|x||W| per output): FP32 accumulation of K <= 864 products of random
sign stays well below that, and one dropped or misplaced term of a 5,000-term
weight-gradient sum is above it.  BF16 outputs must be exactly the RNE
rounding of the FP32 result the kernel wrote beside them.
"""
import numpy as np
import pytest

from oracle import surrogate as so

pytestmark = pytest.mark.gpu

SHAPES = [(2, 5, 16, 32), (1, 3, 8, 16), (1, 4, 24, 48)]
LAYERS = [(8, 32), (32, 32), (32, 8)]


@pytest.fixture(scope="module")
def sur(mpw_lib):
    from paper_2002_00088_gb300 import surrogate
    return surrogate


def torch():
    import torch as t
    return t


def to_dev_bf16(a):
    t = torch()
    return t.from_numpy(so.bf16_bits(a).view(np.int16)).view(t.bfloat16).cuda()


def from_dev(x):
    t = torch()
    if x.dtype == t.bfloat16:
        return so.from_bf16_bits(x.view(t.int16).cpu().numpy().view(np.uint16))
    return x.double().cpu().numpy()


def operands(seed, shape, cin, cout, scale=1.0):
    r = np.random.default_rng(seed)
    x = so.bf16(r.standard_normal(shape + (cin,)) * scale)
    W = so.bf16(r.standard_normal((cout, 27, cin)) / np.sqrt(27 * cin))
    b = r.standard_normal(cout).astype(np.float32).astype(np.float64) * 0.1
    return x, W, b


def assert_bf16_is_rounded_f32(y16, y32):
    np.testing.assert_array_equal(from_dev(y16), so.bf16(from_dev(y32)))


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cin,cout", LAYERS)
@pytest.mark.parametrize("relu", [False, True])
def test_forward_matches_oracle(sur, shape, cin, cout, relu):
    t = torch()
    x, W, b = operands(11 + cin + cout, shape, cin, cout)
    y16, y32 = sur.conv3_forward(to_dev_bf16(x), to_dev_bf16(W), t.tensor(b, dtype=t.float32).cuda(), relu=relu,
                                 out_f32=True)
    want = so.conv3(x, W, b, relu=relu)
    bound = so.conv3(np.abs(x), np.abs(W), np.abs(b))
    err = np.abs(from_dev(y32) - want)
    assert (err <= 2e-5 * bound).all(), err.max()
    assert_bf16_is_rounded_f32(y16, y32)


@pytest.mark.parametrize("cin,cout", LAYERS)
def test_forward_mask_zeroes_outputs(sur, cin, cout):
    x, W, _ = operands(21, (1, 3, 8, 16), cin, cout)
    mask = so.bf16(np.random.default_rng(22).standard_normal((1, 3, 8, 16, cout)))
    _, y32 = sur.conv3_forward(to_dev_bf16(x), to_dev_bf16(W), mask=to_dev_bf16(mask), out_bf16=False, out_f32=True)
    want = np.where(mask > 0, so.conv3(x, W), 0.0)
    err = np.abs(from_dev(y32) - want)
    assert (err <= 2e-5 * so.conv3(np.abs(x), np.abs(W))).all()
    assert (from_dev(y32)[mask <= 0] == 0).all()


@pytest.mark.parametrize("shape", SHAPES[:2])
@pytest.mark.parametrize("cin,cout", LAYERS)
def test_input_gradient_matches_oracle(sur, shape, cin, cout):
    r = np.random.default_rng(31)
    _, W, _ = operands(32, shape, cin, cout)
    gy = so.bf16(r.standard_normal(shape + (cout,)))
    mask = so.bf16(r.standard_normal(shape + (cin,)))
    gx16, gx32 = sur.conv3_backward_data(to_dev_bf16(gy), to_dev_bf16(W), mask=to_dev_bf16(mask), out_f32=True)
    want = so.conv3_input_grad(gy, W, mask)
    bound = so.conv3_input_grad(np.abs(gy), np.abs(W))
    err = np.abs(from_dev(gx32) - want)
    assert (err <= 2e-5 * bound).all(), err.max()
    assert_bf16_is_rounded_f32(gx16, gx32)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("cin,cout", LAYERS)
def test_weight_gradient_matches_oracle(sur, shape, cin, cout):
    t = torch()
    r = np.random.default_rng(41)
    x = so.bf16(r.standard_normal(shape + (cin,)))
    gy = so.bf16(r.standard_normal(shape + (cout,)))
    gw = t.empty((cout, 27, cin), dtype=t.float32, device="cuda")
    gb = t.empty(cout, dtype=t.float32, device="cuda")
    sur.WeightGrad(cin, cout, "cuda")(to_dev_bf16(x), to_dev_bf16(gy), gw, gb)
    want_w, want_b = so.conv3_weight_grad(x, gy)
    bound_w, bound_b = so.conv3_weight_grad(np.abs(x), np.abs(gy))
    err = np.abs(from_dev(gw) - want_w)
    assert (err <= 2e-5 * bound_w).all(), (err / bound_w).max()
    assert (np.abs(from_dev(gb) - want_b) <= 2e-5 * bound_b).all()


def test_weight_gradient_is_deterministic(sur):
    t = torch()
    r = np.random.default_rng(42)
    x = to_dev_bf16(r.standard_normal((2, 6, 16, 32, 32)))
    gy = to_dev_bf16(r.standard_normal((2, 6, 16, 32, 32)))
    wg = sur.WeightGrad(32, 32, "cuda")
    outs = []
    for _ in range(2):
        gw = t.empty((32, 27, 32), dtype=t.float32, device="cuda")
        gb = t.empty(32, dtype=t.float32, device="cuda")
        wg(x, gy, gw, gb)
        outs.append((gw.cpu(), gb.cpu()))
    assert t.equal(outs[0][0], outs[1][0]) and t.equal(outs[0][1], outs[1][1])


def test_adam_matches_oracle(sur):
    """Each step from the device's own state; the oracle takes the binary32
    values of beta1, beta2 and eps that the kernel receives."""
    t = torch()
    r = np.random.default_rng(51)
    n = 10007
    b1, b2, eps = (float(np.float32(c)) for c in (0.9, 0.999, 1e-8))
    dw = t.tensor(r.standard_normal(n).astype(np.float32)).cuda()
    dm = t.zeros(n, dtype=t.float32, device="cuda")
    dv = t.zeros(n, dtype=t.float32, device="cuda")
    w16 = t.empty(n, dtype=t.bfloat16, device="cuda")
    for step in range(1, 4):
        w0, m0, v0 = from_dev(dw), from_dev(dm), from_dev(dv)
        g = (r.standard_normal(n) * 10.0 ** r.uniform(-3, 1, n)).astype(np.float32)
        sur.adam_step(dw, t.tensor(g).cuda(), dm, dv, lr=1e-3, t=step, w16=w16)
        ow, om, ov = so.adam(w0, g.astype(np.float64), m0, v0, 1e-3, b1, b2, eps, step)
        # a few binary32 roundings of each term
        np.testing.assert_array_less(np.abs(from_dev(dm) - om), 1e-6 * (np.abs(m0) + 0.1 * np.abs(g)) + 1e-30)
        np.testing.assert_array_less(np.abs(from_dev(dv) - ov), 1e-6 * (v0 + 1e-3 * g.astype(np.float64) ** 2) + 1e-30)
        np.testing.assert_array_less(np.abs(from_dev(dw) - ow), 1e-6 * np.abs(w0) + 1e-8)
    assert_bf16_is_rounded_f32(w16, dw)


def test_mse_gradient_matches_oracle(sur):
    t = torch()
    r = np.random.default_rng(61)
    P = 4099
    y = r.standard_normal((P, 8)).astype(np.float32)
    tg = r.standard_normal((P, 2)).astype(np.float32)
    gy = t.empty((P, 8), dtype=t.bfloat16, device="cuda")
    loss = t.empty(1, dtype=t.float64, device="cuda")
    sur.mse_grad(t.tensor(y).cuda(), t.tensor(tg).cuda(), gy, loss)
    want_loss, want_g = so.mse(y[:, :2].astype(np.float64), tg.astype(np.float64))
    assert loss.item() == pytest.approx(want_loss, rel=1e-6)
    g = from_dev(gy)
    assert (g[:, 2:] == 0).all()
    # one BF16 rounding of a value that FP32 arithmetic got to within 2 ulp(FP32)
    assert (np.abs(g[:, :2] - want_g) <= np.abs(want_g) * 2.0 ** -8 + 1e-30).all()
