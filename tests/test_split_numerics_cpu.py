"""CPU checks of the split-operand arithmetic the tensor-core path relies on.

Each operand value x (FP32) is scaled by a power of two s that puts max |x s| in [2^10, 2^11)
and split as hi = rn(x s), lo = rn(x s - hi), rn rounding to FP16 (nearest even), BF16
(nearest even) or TF32 (10 explicit mantissa bits in an FP32 word, nearest with ties away from
zero, as cvt.rna.tf32.f32 does).  FP16 and TF32 pairs keep 11 + 11 significant bits, BF16 pairs
8 + 8.  These emulations pin that reading of the mixed forms: a product of split operands
without the lo*lo term is exact to about 2^-22 (FP16, TF32) or 2^-16 (BF16) of |A| |B| per term.
"""
import numpy as np
import pytest


def rn_tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32)
    r = ((b + np.uint32(0x1000)) & np.uint32(0xFFFFE000)).astype(np.uint32)   # magnitude + half ulp
    return r.view(np.float32)


def rn_bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000   # nearest, ties to even
    return r.astype(np.uint32).view(np.float32)


def rn_fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


RN = {"fp16x3": rn_fp16, "bf16x3": rn_bf16, "tf32x3": rn_tf32}
BITS = {"fp16x3": 22, "bf16x3": 16, "tf32x3": 22}


def split(x, prec):
    x = np.asarray(x, dtype=np.float32)
    m = float(np.max(np.abs(x)))
    s = np.float32(2.0 ** (10 - np.floor(np.log2(m)))) if m > 0 else np.float32(1.0)
    xs = x * s                                            # exact: s is a power of two
    hi = RN[prec](xs)
    lo = RN[prec](xs - hi)                                # xs - hi is exact in FP32
    return hi, lo, s


def test_roundings_match_their_definitions():
    # TF32: 10 explicit mantissa bits, ties away from zero; BF16: 7 bits, ties to even
    one = np.float32(1.0)
    ulp_tf32, ulp_bf16 = 2.0 ** -10, 2.0 ** -7
    assert rn_tf32(one + np.float32(ulp_tf32 / 2)) == one + ulp_tf32          # tie: away from zero
    assert rn_tf32(-(one + np.float32(ulp_tf32 / 2))) == -(one + ulp_tf32)
    assert rn_tf32(one + np.float32(ulp_tf32 / 2 - 2.0 ** -23)) == one
    assert rn_bf16(one + np.float32(ulp_bf16 / 2)) == one                      # tie: to even
    assert rn_bf16(one + np.float32(1.5 * ulp_bf16)) == one + 2 * ulp_bf16
    x = np.random.default_rng(1).standard_normal(10000).astype(np.float32)
    for rn, bits in ((rn_tf32, 13), (rn_bf16, 16)):
        r = rn(x).view(np.uint32)
        assert np.all(r & np.uint32((1 << bits) - 1) == 0)                     # dropped bits are zero
        assert np.all(np.abs(rn(x) - x) <= np.abs(x) * 2.0 ** -(24 - bits) * (1 + 1e-6))   # half an ulp


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "tf32x3"])
def test_split_pair_keeps_its_bits(prec):
    # |x s - (hi + lo)| <= 2^-(bits) |x s| for values within FP16's normal range of the scaled max
    rng = np.random.default_rng(7)
    x = rng.uniform(-1.0, 1.0, 20000).astype(np.float32)
    x[np.abs(x) < 1e-3] = 0.5
    hi, lo, s = split(x, prec)
    xs = x.astype(np.float64) * float(s)
    err = np.abs(xs - (hi.astype(np.float64) + lo.astype(np.float64)))
    bound = 2.0 ** -BITS[prec] * np.abs(xs)
    assert np.all(err <= bound), (prec, float(np.max(err / np.abs(xs))))
    # and the bound is tight within a factor of 4 (a dropped lo term would miss it by 2^11)
    assert np.max(err / np.abs(xs)) > 2.0 ** -(BITS[prec] + 2)


@pytest.mark.parametrize("prec", ["fp16x3", "bf16x3", "tf32x3"])
def test_three_product_split_matches_exact_product(prec):
    # C = (A_hi B_hi + A_hi B_lo + A_lo B_hi) / (s_a s_b) in exact arithmetic against A B^T: the
    # dropped lo*lo term and the split residuals leave about 2^-bits of sum |a||b| per entry
    rng = np.random.default_rng(11)
    n = 96
    A = rng.uniform(-1.0, 1.0, (n, n)).astype(np.float32)
    B = rng.uniform(-1.0, 1.0, (n, n)).astype(np.float32)
    ah, al, sa = split(A, prec)
    bh, bl, sb = split(B, prec)
    f = lambda m: m.astype(np.float64)
    C = (f(ah) @ f(bh).T + f(ah) @ f(bl).T + f(al) @ f(bh).T) / (float(sa) * float(sb))
    exact = f(A) @ f(B).T
    scale = np.abs(f(A)) @ np.abs(f(B)).T
    rel = np.max(np.abs(C - exact) / scale)
    assert rel < 2.0 ** -BITS[prec] * 3, (prec, rel)
    # one hi*hi product (the single-product chains) keeps only the hi parts' bits
    C1 = f(ah) @ f(bh).T / (float(sa) * float(sb))
    rel1 = np.max(np.abs(C1 - exact) / scale)
    assert rel1 < 2.0 ** -(BITS[prec] // 2) * 3
    assert rel1 > 2.0 ** 6 * rel                      # the correction segments matter


def test_tf32_and_fp16_pairs_agree_to_their_shared_precision():
    # both keep 22 bits, so their three-product results differ by about 2^-22, while BF16's
    # differs from them by about 2^-16
    rng = np.random.default_rng(3)
    n = 64
    A = rng.uniform(-1.0, 1.0, (n, n)).astype(np.float32)
    B = rng.uniform(-1.0, 1.0, (n, n)).astype(np.float32)
    out = {}
    for prec in RN:
        ah, al, sa = split(A, prec)
        bh, bl, sb = split(B, prec)
        f = lambda m: m.astype(np.float64)
        out[prec] = (f(ah) @ f(bh).T + f(ah) @ f(bl).T + f(al) @ f(bh).T) / (float(sa) * float(sb))
    scale = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64)).T
    d_ft = np.max(np.abs(out["fp16x3"] - out["tf32x3"]) / scale)
    d_fb = np.max(np.abs(out["fp16x3"] - out["bf16x3"]) / scale)
    assert d_ft < 2.0 ** -21
    assert d_fb > 2.0 ** -20
