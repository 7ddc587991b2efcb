"""The tcgen05 (5th-generation tensor core, TMEM accumulator) convolution
kernel that serves volumes 128 points wide, against the numpy oracle
(oracle/surrogate.py) and against the mma.sync kernel (mpw_conv3_select(1)),
element by element.

Bound as in tests/test_gpu_conv.py: FP32 results within 2e-5 of the sum of
the absolute values of the terms; BF16 outputs the RNE rounding of the FP32
ones.  The volumes cover one and several y-chunks of the kernel (16 rows),
a ragged last chunk, the periodic wrap in every direction and a batch of
two; the layers cover the paired-tap first layer (8 -> 32), the 32 -> 32
layers and the last layer with its 8 outputs padded to the MMA's N = 16.
"""
import numpy as np
import pytest

from oracle import surrogate as so
from tests.test_gpu_conv import LAYERS, assert_bf16_is_rounded_f32, from_dev, operands, to_dev_bf16, torch

pytestmark = pytest.mark.gpu

SHAPES_TC = [(1, 3, 8, 128), (2, 4, 24, 128)]


@pytest.fixture(scope="module")
def sur(mpw_lib):
    from paper_2002_00088_gb300 import surrogate
    yield surrogate
    mpw_lib.check(mpw_lib.lib.mpw_conv3_select(0))


@pytest.fixture(params=[0, 1], ids=["tcgen05", "mma_sync"])
def kernel(request, mpw_lib):
    mpw_lib.check(mpw_lib.lib.mpw_conv3_select(request.param))
    yield request.param
    mpw_lib.check(mpw_lib.lib.mpw_conv3_select(0))


@pytest.mark.parametrize("shape", SHAPES_TC)
@pytest.mark.parametrize("cin,cout", LAYERS)
@pytest.mark.parametrize("relu", [False, True])
def test_forward_128_matches_oracle(sur, kernel, shape, cin, cout, relu):
    t = torch()
    x, W, b = operands(71 + cin + cout, shape, cin, cout)
    y16, y32 = sur.conv3_forward(to_dev_bf16(x), to_dev_bf16(W), t.tensor(b, dtype=t.float32).cuda(), relu=relu,
                                 out_f32=True)
    want = so.conv3(x, W, b, relu=relu)
    bound = so.conv3(np.abs(x), np.abs(W), np.abs(b))
    err = np.abs(from_dev(y32) - want)
    assert (err <= 2e-5 * bound).all(), (err / bound).max()
    assert_bf16_is_rounded_f32(y16, y32)


@pytest.mark.parametrize("cin,cout", LAYERS)
def test_forward_128_mask(sur, kernel, cin, cout):
    shape = (1, 3, 24, 128)
    x, W, _ = operands(81, shape, cin, cout)
    mask = so.bf16(np.random.default_rng(82).standard_normal(shape + (cout,)))
    _, y32 = sur.conv3_forward(to_dev_bf16(x), to_dev_bf16(W), mask=to_dev_bf16(mask), out_bf16=False, out_f32=True)
    want = np.where(mask > 0, so.conv3(x, W), 0.0)
    err = np.abs(from_dev(y32) - want)
    assert (err <= 2e-5 * so.conv3(np.abs(x), np.abs(W))).all()
    assert (from_dev(y32)[mask <= 0] == 0).all()


@pytest.mark.parametrize("shape", SHAPES_TC)
@pytest.mark.parametrize("cin,cout", LAYERS)
def test_input_gradient_128_matches_oracle(sur, kernel, shape, cin, cout):
    r = np.random.default_rng(91)
    _, W, _ = operands(92, shape, cin, cout)
    gy = so.bf16(r.standard_normal(shape + (cout,)))
    mask = so.bf16(r.standard_normal(shape + (cin,)))
    gx16, gx32 = sur.conv3_backward_data(to_dev_bf16(gy), to_dev_bf16(W), mask=to_dev_bf16(mask), out_f32=True)
    want = so.conv3_input_grad(gy, W, mask)
    bound = so.conv3_input_grad(np.abs(gy), np.abs(W))
    err = np.abs(from_dev(gx32) - want)
    assert (err <= 2e-5 * bound).all(), (err / bound).max()
    assert_bf16_is_rounded_f32(gx16, gx32)

