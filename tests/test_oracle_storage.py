"""Pins of the oracle's reduced-precision storage emulation: the two software
roundings (binary16, bfloat16; round to nearest, ties to even, IEEE 754) against the
library conversions of numpy and torch, and the emulated step against its definition
(collide, round the stored deviations, stream)."""
import numpy as np
import pytest
import torch

import synth


def _r16(o, xs):
    return np.array([o.round_binary16(x) for x in xs])


def _rbf(o, xs):
    return np.array([o.round_bfloat16(x) for x in xs])


def test_binary16_rounding_matches_numpy(oracle_mod):
    o = oracle_mod.Oracle
    rng = np.random.default_rng(0)
    xs = np.concatenate([
        rng.standard_normal(4000) * np.exp2(rng.integers(-30, 17, 4000)),   # normals, subnormals, overflow
        [0.0, -0.0, 65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 2.0 ** -26],
    ])
    # exact ties between neighbouring binary16 values: (k + 1/2) 2^(E-10) with k in
    # [1024, 2047] for a normal binade E, (k + 1/2) 2^-24 with k < 1024 for subnormals
    for E in (-14, -3, 0, 5, 14):
        k = rng.integers(1024, 2047, 50)
        xs = np.concatenate([xs, (k + 0.5) * 2.0 ** (E - 10), -(k + 0.5) * 2.0 ** (E - 10)])
    k = rng.integers(0, 1023, 50)
    xs = np.concatenate([xs, (k + 0.5) * 2.0 ** -24])
    with np.errstate(over="ignore"):
        want = xs.astype(np.float16).astype(np.float64)
    got = _r16(o, xs)
    np.testing.assert_array_equal(got, want)


def test_bfloat16_rounding_matches_torch(oracle_mod):
    o = oracle_mod.Oracle
    rng = np.random.default_rng(1)
    bits = rng.integers(0, 2 ** 31 - 2 ** 23, 6000, dtype=np.int64).astype(np.uint32)   # finite float32
    bits[::2] |= np.uint32(0x80000000)
    xs = bits.view(np.float32)
    ties = (rng.integers(-2 ** 15, 2 ** 15, 500, dtype=np.int64).astype(np.int32) << 16 | 0x8000).view(np.float32)
    xs = np.concatenate([xs, ties[np.isfinite(ties)], np.float32([1e-40, -3e-39, 3.3e38, -3.39e38])])
    want = torch.from_numpy(xs).to(torch.bfloat16).to(torch.float64).numpy()
    got = _rbf(o, xs.astype(np.float64))
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("mode,bits", [("f16s", 11), ("bf16s", 8)])
def test_emulated_step_is_collide_round_stream(oracle_mod, mode, bits):
    n, r, s = (10, 8, 6), 0.5, 1.0
    kw = dict(r=r, s=s, omega_nu=1.4, omega_xi=1.0, walls="y", force=(1e-5, 0.0, 0.0))
    oq = oracle_mod.Oracle(*n, storage_emulation=mode, **kw)
    op = oracle_mod.Oracle(*n, **kw)
    rho, u = synth.solenoidal_random(*n, r, s, 2.0, 0.03, seed=9)
    f0p = op.init(rho, u)
    f0 = oq.init(rho, u)
    np.testing.assert_array_equal(f0, oq.quantize(f0p))
    np.testing.assert_array_equal(oq.quantize(f0), f0)                  # idempotent
    w = op.equilibrium(1.0, np.zeros(3))
    g, gp = f0 - w[:, None, None, None], f0p - w[:, None, None, None]
    # at most half a unit in the last place of the stored format (relative to g)
    assert np.all(np.abs(g - gp) <= np.abs(gp) * 2.0 ** -bits + 1e-300)
    f1 = oq.step(f0)
    np.testing.assert_array_equal(f1, op.stream(oq.quantize(op.collide_all(f0))))
    assert not np.array_equal(f1, op.step(f0))                          # the rounding does act
