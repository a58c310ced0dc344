"""Pins of the oracle's canonical distance to closed forms (CPU only).

The paper uses ||x_v - x_w|| (Algorithm 2) without fixing precision; the
oracle's reading is a squared fp32 distance with one fixed operation order.
These tests tie it to exact arithmetic, not to itself.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore")


def test_integer_inputs_are_exact(oracle_mod):
    # Integer coordinates in 0..255, m = 128: every partial sum is an integer
    # below 2^24, so the fp32 result must equal the exact integer sum.
    rng = np.random.default_rng(1)
    for m in (4, 37, 96, 128):
        for _ in range(50):
            a = rng.integers(0, 256, m)
            b = rng.integers(0, 256, m)
            exact = int(((a - b) ** 2).sum())
            got = oracle_mod.dist(a.astype(np.float32), b.astype(np.float32))
            assert got == float(exact)


def test_relative_error_against_fp64(oracle_mod):
    # fp32 fused multiply-add chains of length <= m/128 * 4 and a 5-level tree:
    # the error bound is far inside 1e-5 relative for m <= 960.
    rng = np.random.default_rng(2)
    for m in (96, 128, 768, 960, 1001):
        for _ in range(20):
            a = rng.normal(0, 10, m).astype(np.float32)
            b = (a + rng.normal(0, 1, m)).astype(np.float32)
            d32 = oracle_mod.dist(a, b)
            d64 = float(((a.astype(np.float64) - b.astype(np.float64)) ** 2).sum())
            assert abs(d32 - d64) <= 1e-5 * d64


def test_inner_product_form(oracle_mod):
    rng = np.random.default_rng(3)
    for m in (96, 768):
        a = rng.normal(size=m); a /= np.linalg.norm(a)
        b = rng.normal(size=m); b /= np.linalg.norm(b)
        a, b = a.astype(np.float32), b.astype(np.float32)
        got = oracle_mod.dist(a, b, "ip")
        ref = 1.0 - float(np.dot(a.astype(np.float64), b.astype(np.float64)))
        assert abs(got - ref) <= 1e-6
        # exact special case: orthogonal basis vectors give 1, identical give 0
        e0 = np.zeros(m, np.float32); e0[0] = 1
        e1 = np.zeros(m, np.float32); e1[5] = 1
        assert oracle_mod.dist(e0, e1, "ip") == 1.0
        assert oracle_mod.dist(e0, e0, "ip") == 0.0


def test_symmetry_and_identity(oracle_mod):
    rng = np.random.default_rng(4)
    for m in (128, 960):
        a = rng.normal(0, 10, m).astype(np.float32)
        b = rng.normal(0, 10, m).astype(np.float32)
        assert oracle_mod.dist(a, b) == oracle_mod.dist(b, a)
        assert oracle_mod.dist(a, b, "ip") == oracle_mod.dist(b, a, "ip")
        assert oracle_mod.dist(a, a) == 0.0


def test_zero_padding_is_neutral(oracle_mod):
    # Rows stored with zero padding to a multiple of 4 (or of 128) must give
    # the same bits: appended zeros add fma(0, 0, acc) = acc to their partial.
    rng = np.random.default_rng(5)
    for m in (37, 95, 130):
        a = rng.normal(0, 3, m).astype(np.float32)
        b = rng.normal(0, 3, m).astype(np.float32)
        pad = (-m) % 128
        ap = np.concatenate([a, np.zeros(pad, np.float32)])
        bp = np.concatenate([b, np.zeros(pad, np.float32)])
        assert oracle_mod.dist(a, b) == oracle_mod.dist(ap, bp)
        assert oracle_mod.dist(a, b, "ip") == oracle_mod.dist(ap, bp, "ip")


def test_order_dependence_is_real(oracle_mod):
    # Guard that the pins above are not vacuous: a different summation order
    # (plain sequential fp32) differs from the canonical tree on some inputs.
    rng = np.random.default_rng(6)
    diffs = 0
    for _ in range(200):
        a = rng.normal(0, 10, 128).astype(np.float32)
        b = rng.normal(0, 10, 128).astype(np.float32)
        seq = np.float32(0)
        for x, y in zip(a, b):
            t = np.float32(x - y)
            seq = np.float32(seq + np.float32(t * t))
        diffs += oracle_mod.dist(a, b) != float(seq)
    assert diffs > 0
