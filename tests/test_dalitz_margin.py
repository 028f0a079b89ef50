"""The FP32 Dalitz-plot check of the CUDA path decides an event in FP32 only
outside a margin derived from its rounding errors, and sends the rest to an
FP64 test. This file checks that derivation on the CPU: a float32 emulation of
both FP32 stages (every operation rounded to float32 as on the GPU, the
hardware 1/sqrt perturbed by up to its 2^-22.9 relative error), on points
placed 1e-9 .. 1e-3 (relative) off the boundary and on uniform points, must
never decide differently from the oracle's FP64 boundary test, and must send
only a small fraction of uniform events to the FP64 test.

The emulation restates the kernel's formulas (stage 1: the square-root-free
form G = 4 l1 l3 - A^2 with a 2^-18 bound; stage 2: lo <= s23 <= hi with the
3e-6 / 2e-6 margins); it is test code, not a copy of the device code path.
"""
import numpy as np
import pytest

import synth
from tests import _problems as P

f = np.float32


def _near_boundary(spec, n, rng):
    m1, m2, mD = spec.m1, spec.m2, spec.mD
    smin, smax = (m1 + m2) ** 2, (mD - m2) ** 2
    t = np.concatenate([rng.uniform(smin, smax, n // 2),
                        smin * (1 + 10 ** rng.uniform(-7, -1, n // 4)),
                        smax * (1 - 10 ** rng.uniform(-7, -1, n - n // 2 - n // 4))])
    e2 = (t - m1 * m1 + m2 * m2) / (2 * np.sqrt(t))
    e3 = (mD * mD - t - m2 * m2) / (2 * np.sqrt(t))
    k2 = np.sqrt(np.maximum(e2 * e2 - m2 * m2, 0))
    k3 = np.sqrt(np.maximum(e3 * e3 - m2 * m2, 0))
    es = (e2 + e3) ** 2
    b = np.where(rng.random(n) < 0.5, es - (k2 + k3) ** 2, es - (k2 - k3) ** 2)
    b = b * (1 + rng.choice([-1, 1], n) * 10 ** rng.uniform(-9, -3, n))
    s13 = (mD * mD + m1 * m1 + 2 * m2 * m2) - t - b
    return np.stack([np.concatenate([t, s13]), np.concatenate([s13, t])], axis=1)


def _fp32_decision(spec, s12, s13, rng):
    """(decided inside, decided outside) of the two FP32 stages, emulated."""
    m1, m2, mD = spec.m1, spec.m2, spec.mD
    thr_p, pthr_m = f((m1 + m2) ** 2), f((mD - m2) ** 2)
    m1s, m2s, mDs = f(m1 * m1), f(m2 * m2), f(mD * mD)
    sigma = f(mD * mD + m1 * m1 + 2 * m2 * m2)
    s12, s13 = s12.astype(f), s13.astype(f)
    tol = f(1e-4)
    clear = ((s12 > thr_p * (f(1) + tol)) & (s12 < pthr_m * (f(1) - tol)) &
             (s13 > thr_p * (f(1) + tol)) & (s13 < pthr_m * (f(1) - tol)))
    s23 = (sigma - s12) - s13
    # stage 1
    q = f(4) * s12 * m2s
    a1 = (s12 - m1s) + m2s
    a3 = (mDs - s12) - m2s
    l1, l3 = a1 * a1 - q, a3 * a3 - q
    d = mDs - m1s
    A = ((f(4) * s12 * s23 - d * d) + l1) + l3
    G = f(4) * l1 * l3 - A * A
    a1m, a3m = (s12 + m1s) + m2s, (mDs + s12) + m2s
    l1m, l3m = a1m * a1m + q, a3m * a3m + q
    dm = mDs + m1s
    Am = ((f(4) * s12 * ((sigma + s12) + s13) + dm * dm) + l1m) + l3m
    err = f(2.0 ** -18) * (Am * Am + f(4) * l1m * l3m)
    in1, out1 = clear & (G > err), clear & (G < -err)
    # stage 2 (the hardware 1/sqrt: up to 2^-22.9 relative error)
    r = (f(1) / np.sqrt(s12)) * (f(1) + f(2.0 ** -22.9) * rng.uniform(-1, 1, s12.shape).astype(f))
    inv2 = f(0.5) * r
    e2, e3 = ((s12 - m1s) + m2s) * inv2, ((mDs - s12) - m2s) * inv2
    k2 = np.sqrt(np.maximum(e2 * e2 - m2s, f(0)))
    k3 = np.sqrt(np.maximum(e3 * e3 - m2s, f(0)))
    es = (e2 + e3) * (e2 + e3)
    kk = (k2 + k3) * (k2 + k3)
    lo, hi = es - kk, es - (k2 - k3) * (k2 - k3)
    e2m, e3m = ((s12 + m1s) + m2s) * inv2, ((mDs + s12) + m2s) * inv2
    w2, w3 = e2m * e2m + m2s, e3m * e3m + m2s
    with np.errstate(divide="ignore", invalid="ignore"):
        mg = (f(3e-6) * ((e2m + e3m) * (e2m + e3m) + kk + ((sigma + s12) + s13)) +
              f(2e-6) * (k2 + k3) * (w2 / k2 + w3 / k3))
        in2 = clear & (s23 > lo + mg) & (s23 < hi - mg)
        out2 = clear & ((s23 < lo - mg) | (s23 > hi + mg))
    first = in1 | out1
    return in1 | (~first & in2), out1 | (~first & out2), clear


@pytest.mark.parametrize("name", ["pipipi_n10", "kpipi_n40", "kkk_n40"])
def test_fp32_dalitz_decisions_agree_with_fp64(name):
    spec = P.spec_by_name(name)
    o = P.oracle_for(name)
    rng = np.random.default_rng(77)
    near = _near_boundary(spec, 300_000, rng).astype(np.float32).astype(np.float64)
    lo, hi = spec.s_lo, spec.s_hi
    uni = (lo + (hi - lo) * rng.random((600_000, 2))).astype(np.float32).astype(np.float64)
    for pts, max_fallback in ((near, 1.0), (uni, 1e-3)):
        ref = o.inside(pts).astype(bool)
        din, dout, clear = _fp32_decision(spec, pts[:, 0], pts[:, 1], rng)
        assert not np.any(din & ~ref), "decided inside, outside in FP64"
        assert not np.any(dout & ref), "decided outside, inside in FP64"
        fallback = clear & ~(din | dout)
        assert fallback.mean() <= max_fallback, fallback.mean()
