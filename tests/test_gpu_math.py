"""The FP32 step's hand-written forms against the exact values and against CUDA's own functions.

The paired FP32 step replaces library calls by forms of its own: 1/d (d >= 1) by the
hardware reciprocal estimate refined by one Newton-Raphson step; the carrier-phase sine and
cosine by a Cody-Waite reduction by 2 pi followed by the hardware sine and cosine; the
probability 1 - e^-x of Eq. 4 by a four-term Taylor series below 2^-5; and, for the 2D focus,
the amplitude and Gouy phase (1 + a^2)^(-1/4) e^{i atan(a)/2} by the half-angle square root of
1 + i a, and the transverse profile e^{-y^2/w^2} by the hardware base-2 exponential.  pe_math_probe runs the
very device functions the step uses; here they are swept over the ranges the step feeds them
and compared with the exact values (FP64 on the host, of the same float inputs), with the
error bounds the design states, and with CUDA's __frcp_rn, sinf, cosf and expm1f.
"""
import math

import numpy as np
import pytest

import paper_1612_07592_gb300 as pe

pytestmark = pytest.mark.gpu
M = pe.PE_MATH


def probe(fn, x):
    import torch
    xin = torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).cuda()
    out = torch.empty_like(xin)
    s = torch.cuda.current_stream()
    pe.pe_math_probe(fn, xin.data_ptr(), out.data_ptr(), xin.numel(), s.cuda_stream)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64)


def ulp(v):
    """Spacing of floats at |v| (normal range)."""
    e = np.floor(np.log2(np.abs(v)))
    return np.ldexp(1.0, (e - 23).astype(int))


def test_reciprocal_within_one_ulp():
    rng = np.random.default_rng(1)
    d = np.concatenate([np.exp(rng.uniform(0.0, math.log(1e5), 1 << 20)),
                        1.0 + rng.uniform(0.0, 1.0, 1 << 18), np.array([1.0, 2.0, 3.0, 1e5])]).astype(np.float32)
    exact = 1.0 / d.astype(np.float64)
    ours = probe(M["RCP"], d)
    cuda = probe(M["CUDA_RCP"], d)
    e_ours = np.abs(ours - exact) / ulp(exact)
    e_cuda = np.abs(cuda - exact) / ulp(exact)
    print(f"rcp: max {e_ours.max():.3f} ulp (CUDA __frcp_rn {e_cuda.max():.3f}), "
          f"{np.mean(ours != cuda):.4f} of results differ from the correctly rounded one")
    assert e_cuda.max() <= 0.5 + 1e-9
    assert e_ours.max() <= 1.0


@pytest.mark.parametrize("lo,hi,bound_log2", [(-math.pi, math.pi, -21.2), (-400.0, 400.0, -20.9)])
def test_phase_sine_cosine(lo, hi, bound_log2):
    """[-pi, pi]: the hardware sine and cosine alone, measured on GB300 at 2^-21.48 (sine) and
    2^-21.25 (cosine) over this sweep, bound 2^-21.2; [-400, 400] covers the phases t - x and
    t + x - 2 x_m of 4000 steps of T/100: the reduced argument is rounded once (half an ulp of a
    value below pi, 2^-23), measured 2^-20.98, bound 2^-20.9.  CUDA's sinf and cosf stay near
    2^-23.5; the field error this leaves, a0 x 5e-7, is far below the FP32 rounding of the
    momenta."""
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.uniform(lo, hi, 1 << 21), np.linspace(lo, hi, 1 << 16)]).astype(np.float32)
    vd = v.astype(np.float64)
    s, c = probe(M["SIN"], v), probe(M["COS"], v)
    np.testing.assert_array_equal(s, probe(M["SIN1"], v))       # paired and one-electron forms agree
    np.testing.assert_array_equal(c, probe(M["COS1"], v))
    es, ec = np.abs(s - np.sin(vd)).max(), np.abs(c - np.cos(vd)).max()
    cs = np.abs(probe(M["CUDA_SIN"], v) - np.sin(vd)).max()
    cc = np.abs(probe(M["CUDA_COS"], v) - np.cos(vd)).max()
    print(f"[{lo:g}, {hi:g}]: sin {math.log2(es):.2f}, cos {math.log2(ec):.2f} (log2 abs error); "
          f"CUDA sinf {math.log2(cs):.2f}, cosf {math.log2(cc):.2f}")
    assert max(es, ec) < 2.0 ** bound_log2


def test_brems_probability_series():
    rng = np.random.default_rng(3)
    x = np.concatenate([np.exp(rng.uniform(math.log(1e-10), math.log(2.0 ** -5), 1 << 20)),
                        rng.uniform(2.0 ** -5, 1.0, 1 << 16)]).astype(np.float32)
    exact = -np.expm1(-x.astype(np.float64))
    ours = probe(M["BREMS_P"], x)
    np.testing.assert_array_equal(ours, probe(M["BREMS_P1"], x))  # paired and one-electron forms agree
    cuda = probe(M["CUDA_EXPM1"], x)
    rel = np.abs(ours - exact) / exact
    relc = np.abs(cuda - exact) / exact
    small = x < 2.0 ** -5
    print(f"1 - e^-x: series max rel {rel[small].max():.3g} (expm1f {relc[small].max():.3g}); "
          f"above 2^-5 {rel[~small].max():.3g}")
    assert rel[small].max() < 1.0e-7
    np.testing.assert_array_equal(ours[~small], cuda[~small])


def test_gouy_factors():
    """(1 + a^2)^(-1/4) cos(atan(a)/2) and ... sin(...) against FP64: a over the distances from
    the focus a run reaches (|a| < 1 in the 2D workloads) and beyond; the forms use two hardware
    reciprocal square roots and a few roundings: measured on GB300 2^-21.8 (cos part) and 2^-23.7
    (sin part) absolute, bound 2^-21 (the values are below 1)."""
    rng = np.random.default_rng(4)
    a = np.concatenate([rng.uniform(-1.0, 1.0, 1 << 20), rng.uniform(-50.0, 50.0, 1 << 16),
                        np.array([0.0, 1e-6, -1e-6, 1.0, -1.0])]).astype(np.float32)
    ad = a.astype(np.float64)
    amp = (1.0 + ad * ad) ** -0.25
    ec = np.abs(probe(M["GOUY_C"], a) - amp * np.cos(0.5 * np.arctan(ad))).max()
    es = np.abs(probe(M["GOUY_S"], a) - amp * np.sin(0.5 * np.arctan(ad))).max()
    print(f"Gouy factors: cos part {math.log2(ec):.2f}, sin part {math.log2(es):.2f} (log2 abs error)")
    assert max(ec, es) < 2.0 ** -21


def test_transverse_profile_exponential():
    """e^-v for 0 <= v <= 30 against FP64: the hardware base-2 exponential of -v log2(e); the
    product v log2(e) is rounded once, which adds about v 2^-24 relative: measured on GB300 1.6e-7
    relative for v <= 1 and 1.7e-6 up to v = 30, bound 2^-21 (1 + v)."""
    rng = np.random.default_rng(5)
    v = np.concatenate([rng.uniform(0.0, 1.0, 1 << 20), rng.uniform(0.0, 30.0, 1 << 18),
                        np.array([0.0, 1e-30, 1.0])]).astype(np.float32)
    vd = v.astype(np.float64)
    exact = np.exp(-vd)
    rel = np.abs(probe(M["EXP_NEG"], v) - exact) / exact
    print(f"e^-v: max rel {rel.max():.3g}, over v <= 1 {rel[vd <= 1.0].max():.3g}")
    assert np.all(rel < 2.0 ** -21 * (1.0 + vd))


def tau_exact(lo, hi):
    """-ln U for U = (the top 53 bits of hi:lo + 1/2) / 2^53, to 40 digits."""
    from decimal import Decimal, localcontext
    with localcontext() as ctx:
        ctx.prec = 40
        b = ((int(hi) << 32) | int(lo)) >> 11
        return float(-((Decimal(b) + Decimal("0.5")) / Decimal(2 ** 53)).ln())


def tau_words():
    """Random 64-bit words plus the edges of the form: U below 2^-23 (the high float is 0),
    just above it and around the renormalisation at 2^-10, around 1/2 (the complement branch
    starts at the top bit), and U within 2^-23 of 1."""
    rng = np.random.default_rng(7)
    w = rng.integers(0, 1 << 32, size=(1 << 14, 2), dtype=np.uint64)
    edges = [(lo, hi) for hi in (0, 1, 0x1FF, 0x200, 0x201, 0x3FF, 0x2FF, 0x7FF, 0x1FFF, 0x3FFFFF, 0x400000,
                                 0x7FFFFFFF, 0x80000000, 0x80000001, 0xFFFFFE00, 0xFFFFFFFE, 0xFFFFFFFF)
             for lo in (0, 0x7FF, 0x800, 0x12345678, 0xFFFFF800, 0xFFFFFFFF)]
    return np.concatenate([w, np.array(edges, dtype=np.uint64)])


def test_optical_depth_draw():
    """The FP32 optical depth -ln U (the draw after every emission) against 40-digit logarithms
    of the same 53-bit U, over random words and the edges of the form: relative error measured
    2^-22.91 on GB300 (2^-22.75 in the float32 emulation of the form on the host), bound 2^-21.5.  Before the renormalisation of
    the pair below U = 2^-10 the form gave NaN for U < 2^-23 (about one draw in 8.4e6) and
    first-order errors of several per cent just above."""
    import torch
    w = tau_words()
    words = np.empty(2 * len(w), dtype=np.uint32)
    words[0::2] = w[:, 0]
    words[1::2] = w[:, 1]
    xin = torch.from_numpy(words.view(np.float32)).cuda()
    out = torch.empty(len(w), dtype=torch.float32, device="cuda")
    pe.pe_math_probe(M["TAU"], xin.data_ptr(), out.data_ptr(), len(w), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    ours = out.cpu().numpy().astype(np.float64)
    exact = np.array([tau_exact(lo, hi) for lo, hi in w])
    assert np.all(np.isfinite(ours)) and np.all(ours > 0)
    rel = np.abs(ours - exact) / exact
    print(f"tau: max relative error 2^{math.log2(rel.max()):.2f}")
    assert rel.max() <= 2.0 ** -21.5
