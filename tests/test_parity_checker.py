"""CPU checks of the population-level parity check used by the tensor-core
learned-collision GPU tests (tests/gpu_helpers.learned_pop_check): it accepts
the oracle's own result at FP32 rounding and bf16 activation-rounding level,
and rejects results with the network or a part of it missing (mistakes planted
in the oracle's inputs, on the CPU)."""
import numpy as np
import pytest

import oracle
from paper_2403_18466_gb300 import inputs
from gpu_helpers import bf16_round, learned_pop_check, learned_theta, population_field

ALPHA = 5e-2  # the tolerance factor of tests/test_gpu_mlp_bf16.py


@pytest.fixture(scope="module")
def case():
    theta = learned_theta(5)
    thb = bf16_round(theta)
    f = population_field(1, 16, 24, seed=3).astype(np.float64)
    g = oracle.stream_push(f)
    prm = oracle.params(0.6, force_amp=1e-4, force_mode=1)
    ref = oracle.step(oracle.MLP, g, prm, thb)
    ref_bgk = oracle.step(oracle.BGK, g, prm)
    return theta, thb, g, prm, ref, ref_bgk


def test_accepts_the_reference_at_fp32_rounding(case):
    _, _, _, _, ref, ref_bgk = case
    ok, err, corr, tol = learned_pop_check(ref.astype(np.float32), ref, ref_bgk, ALPHA)
    assert ok and err < 1e-6 * corr


def test_accepts_bf16_weight_rounding_level(case):
    """The unrounded-weight result differs from the bf16-weight one by the
    weight rounding only (~2e-3 of the correction): inside the tolerance."""
    theta, _, g, prm, ref, ref_bgk = case
    ok, err, corr, _ = learned_pop_check(oracle.step(oracle.MLP, g, prm, theta), ref, ref_bgk,
                                         ALPHA)
    assert ok and 1e-4 * corr < err < 1e-2 * corr


def _mutated(thb, which):
    th = thb.copy()
    W1, b1, W2, b2, W3, b3 = inputs.unpack_mlp(th)
    if which == "no_output_layer":
        W3[:] = 0.0
        b3[:] = 0.0
    elif which == "no_hidden_biases":
        b1[:] = 0.0
        b2[:] = 0.0
    elif which == "output_sign":
        W3 *= -1.0
        b3 *= -1.0
    elif which == "second_layer_transposed":
        W2[:] = W2.T.copy()
    elif which == "first_layer_rows_swapped":
        W1[:] = W1[::-1].copy()
    elif which == "input_ignored":
        W1[:] = 0.0
    elif which == "input_doubled":
        W1 *= 2.0
    return th


@pytest.mark.parametrize("which", ["no_output_layer", "no_hidden_biases", "output_sign",
                                   "second_layer_transposed", "first_layer_rows_swapped",
                                   "input_ignored", "input_doubled"])
def test_rejects_planted_mistakes(case, which):
    _, thb, g, prm, ref, ref_bgk = case
    bad = oracle.step(oracle.MLP, g, prm, _mutated(thb, which))
    ok, err, corr, tol = learned_pop_check(bad, ref, ref_bgk, ALPHA)
    assert not ok, (which, err, corr)


def test_rejects_plain_bgk(case):
    _, _, _, _, ref, ref_bgk = case
    ok, err, corr, _ = learned_pop_check(ref_bgk, ref, ref_bgk, ALPHA)
    assert not ok and err == corr
