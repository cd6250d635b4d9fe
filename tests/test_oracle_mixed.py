"""Pins for oracle.mixed: rounding helpers and the identity-rounding limit."""
import numpy as np
import pytest

from oracle import mixed
from oracle.fd import FD
from oracle.system import STProblem


def test_round_bf16_bit_patterns():
    # 1 + 2^-8 is halfway between bf16 neighbours 1 and 1 + 2^-7: ties to even -> 1
    assert mixed.round_bf16(np.float32(1 + 2 ** -8)) == np.float32(1.0)
    # 1 + 3 * 2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6: ties to even -> 1 + 2^-6
    assert mixed.round_bf16(np.float32(1 + 3 * 2 ** -8)) == np.float32(1 + 2 ** -6)
    assert mixed.round_bf16(np.float32(1 + 2 ** -8 + 2 ** -12)) == np.float32(1 + 2 ** -7)
    assert mixed.round_bf16(np.float32(-3.0)) == np.float32(-3.0)
    x = np.random.default_rng(0).standard_normal(1000).astype(np.float32)
    rel = np.abs(mixed.round_bf16(x) - x) / np.abs(x)
    assert rel.max() <= 2.0 ** -8 * (1 + 1e-6)


def test_round_tf32_bit_patterns():
    # ties away from zero at 10 mantissa bits
    assert mixed.round_tf32(np.float32(1 + 2 ** -11)) == np.float32(1 + 2 ** -10)
    assert mixed.round_tf32(np.float32(-(1 + 2 ** -11))) == np.float32(-(1 + 2 ** -10))
    assert mixed.round_tf32(np.float32(1 + 2 ** -12)) == np.float32(1.0)
    x = np.random.default_rng(1).standard_normal(1000).astype(np.float32)
    assert (np.abs(mixed.round_tf32(x) - x) / np.abs(x)).max() <= 2.0 ** -11 * (1 + 1e-6)


def test_mixed_model_close_to_fp64_and_ordered():
    prob = STProblem(2, 3, 6)
    fd = FD(prob)
    r = np.random.default_rng(2).uniform(-1, 1, prob.N)
    z = fd.apply(r)
    e_bf = np.linalg.norm(mixed.apply_mixed(fd, r, "bf16") - z) / np.linalg.norm(z)
    e_tf = np.linalg.norm(mixed.apply_mixed(fd, r, "tf32") - z) / np.linalg.norm(z)
    assert e_tf < e_bf < 5e-2
    assert e_tf < 5e-3


@pytest.mark.parametrize("bwd_order", ["ascending", "descending"])
def test_identity_rounding_is_algorithm_1(bwd_order):
    prob = STProblem(3, 2, 3)
    fd = FD(prob)
    r = np.random.default_rng(4).uniform(-1, 1, prob.N)
    np.testing.assert_allclose(mixed.apply_mixed(fd, r, "fp64", bwd_order), fd.apply(r), rtol=1e-13, atol=1e-14)


def test_backward_order_changes_only_roundings():
    """Both orders are Algorithm 1 with different rounding points: their BF16 results
    differ from each other by about the model's own rounding error, and each is within
    the BF16 bound of the exact solve."""
    prob = STProblem(2, 3, 5)
    fd = FD(prob)
    r = np.random.default_rng(5).uniform(-1, 1, prob.N)
    z = fd.apply(r)
    za = mixed.apply_mixed(fd, r, "bf16", "ascending")
    zd = mixed.apply_mixed(fd, r, "bf16", "descending")
    ea = np.linalg.norm(za - z) / np.linalg.norm(z)
    ed = np.linalg.norm(zd - z) / np.linalg.norm(z)
    assert ea < 5e-2 and ed < 5e-2
    assert 0 < np.linalg.norm(za - zd) / np.linalg.norm(z) < 5e-2
    with pytest.raises(ValueError):
        mixed.apply_mixed(fd, r, "bf16", "sideways")
