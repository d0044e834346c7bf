"""The bf16 sketch's rounding decision, emulated on the CPU (no GPU, no CUDA code).

The kernel rounds each normalised sample to bfloat16 from float32 arithmetic:
v = ((x - mu_hi) - mu_lo) * r32, an error bound E = 2^-21 |v| + 2^-46 r |mu|
+ 2^-125, and the decision is taken only when v - E (rounded down) and v + E
(rounded up) round to the same bfloat16; otherwise the float64 value is
rounded.  Here numpy float32 arithmetic (nearest) and directed rounding of the
exact float64 sums reproduce those steps, and every decision the float32 path
takes must equal the oracle's nearest-even bfloat16 of (x - mu) / sigma.  Half
of the samples are placed next to bfloat16 rounding midpoints.  A control with
a bound too small must produce wrong decisions, so the check can fail.
"""
import numpy as np
import pytest

from oracle import tsk_oracle as o


def _rd32(z):
    f = z.astype(np.float32)
    lower = f.astype(np.float64) > z
    f[lower] = np.nextafter(f[lower], np.float32(-np.inf))
    return f


def _ru32(z):
    f = z.astype(np.float32)
    higher = f.astype(np.float64) < z
    f[higher] = np.nextafter(f[higher], np.float32(np.inf))
    return f


def _bf16_rn_bits(f32):
    """Nearest-even bfloat16 bits of float32 values (cvt.rn.bf16 of a float32)."""
    b = f32.view(np.uint32).astype(np.uint64)
    return ((b + np.uint64(0x7FFF) + ((b >> np.uint64(16)) & np.uint64(1))) >> np.uint64(16)).astype(np.uint32)


def _decisions(x, mu, sigma, coef, cscale):
    r = 1.0 / sigma
    muh = np.float32(mu)
    mul = np.float32(mu - float(muh))
    rh = np.float32(r)
    c0 = np.float32(cscale * (2.0 ** -46 * r * abs(mu) + 2.0 ** -125) * 1.001)
    v = ((x + (-muh)) + (-mul)) * rh                                   # float32, nearest
    e = (np.abs(v).astype(np.float64) * coef + float(c0)).astype(np.float32)
    lo = _rd32(v.astype(np.float64) - e.astype(np.float64))
    hi = _ru32(v.astype(np.float64) + e.astype(np.float64))
    blo, bhi = _bf16_rn_bits(lo), _bf16_rn_bits(hi)
    decided = blo == bhi
    ref = o.bf16_round((x.astype(np.float64) - mu) / sigma).astype(np.float32).view(np.uint32) >> np.uint32(16)
    return decided, blo, ref


def _samples(rng, mu, sigma, n):
    w = rng.normal(size=n) * 2
    mids = ((w.astype(np.float32).view(np.uint32) & np.uint32(0xFFFF0000)) | np.uint32(0x8000)).view(np.float32)
    w = np.where(rng.random(n) < 0.5, w, mids.astype(np.float64) * (1 + rng.normal(size=n) * 1e-7))
    return (mu + w * sigma).astype(np.float32)


@pytest.mark.parametrize("mu,sigma", [(0.0, 1.0), (0.37, 3.3), (1e4, 1.0), (-2.5e6, 37.0), (123.456, 3e-6), (1e-3, 1e5)])
def test_float32_decisions_equal_the_float64_rounding(mu, sigma):
    rng = np.random.default_rng(int(abs(mu) * 7 + sigma * 11) % 2**32)
    x = _samples(rng, mu, sigma, 400000)
    decided, got, ref = _decisions(x, mu, sigma, 2.0 ** -21, 1.0)
    assert decided.mean() > 0.45                   # all but the samples placed on top of midpoints
    assert np.array_equal(got[decided], ref[decided])


@pytest.mark.parametrize("mu,sigma", [(0.37, 3.3), (1.7, 0.3)])
def test_a_bound_too_small_decides_wrongly(mu, sigma):
    """Control: with E = 2^-27 |v| (below the float32 error) some decisions are wrong."""
    rng = np.random.default_rng(5)
    x = _samples(rng, mu, sigma, 400000)
    decided, got, ref = _decisions(x, mu, sigma, 2.0 ** -27, 0.0)
    assert (got[decided] != ref[decided]).sum() > 100
    # and the kernel's bound on the same samples decides every one of them right
    decided, got, ref = _decisions(x, mu, sigma, 2.0 ** -21, 1.0)
    assert np.array_equal(got[decided], ref[decided])
