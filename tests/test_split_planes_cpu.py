"""The arithmetic the mixed exchange relies on, checked on the CPU with numpy (no GPU, no
library): the row-scaled BF16 planes and the exactness of the fixed-point products' sums in
FP32.  The kernels' results are compared with the same emulation in test_gpu_mixed.py."""
import numpy as np


def bf16_rn(x):
    m, e = np.frexp(np.asarray(x, dtype=np.float64))
    return np.ldexp(np.round(m * 256.0), e - 8)


def planes(x, n=5):
    amax = np.max(np.abs(x))
    sig = np.ldexp(1.0, np.frexp(amax)[1]) if amax > 0 else 0.0
    out, r = [], x.copy()
    for g in (128.0, 32768.0):
        h = np.round(r * g / sig) * sig / g if sig > 0 else np.zeros_like(r)
        out.append(h)
        r = r - h
    for _ in range(n - 2):
        q = bf16_rn(r)
        out.append(q)
        r = r - q
    return sig, out, r


def test_fixed_point_planes_are_small_integers_on_row_grids():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(4096) * np.exp(rng.uniform(-20, 0, 4096))   # 9 decades below the max
    sig, p, _ = planes(x)
    q0, q1 = p[0] * 128.0 / sig, p[1] * 32768.0 / sig
    assert np.all(q0 == np.round(q0)) and np.max(np.abs(q0)) <= 128
    assert np.all(q1 == np.round(q1)) and np.max(np.abs(q1)) <= 128
    for pl in p:                                   # every plane is exactly a BF16 value
        assert np.array_equal(bf16_rn(pl), pl)


def test_five_planes_reconstruct_to_2e_minus_40_of_the_row_max_and_24_bits_of_each_element():
    rng = np.random.default_rng(1)
    x = rng.standard_normal(4096) * np.exp(rng.uniform(-20, 0, 4096))
    sig, p, r = planes(x)
    assert np.max(np.abs(r)) <= 2.0 ** -40 * sig
    assert np.all(np.abs(r) <= 2.0 ** -24 * np.abs(x) + 2.0 ** -40 * sig)


def test_fixed_point_products_sum_exactly_in_fp32():
    """Products of two p0 rows are integers times one scale: the FP32 running sum of 256 of
    them (|q| <= 128) never leaves the 24-bit integer range, so it is exact; the same sum of
    per-element BF16 values is not."""
    rng = np.random.default_rng(2)
    a = rng.standard_normal(256)
    b = rng.standard_normal(256)
    sa, pa, _ = planes(a)
    sb, pb, _ = planes(b)
    qa, qb = pa[0] * 128.0 / sa, pb[0] * 128.0 / sb
    acc = np.float32(0.0)
    for u, v in zip(qa, qb):
        acc = np.float32(acc + np.float32(u * v))
    assert float(acc) == float(np.dot(qa, qb))
    ha, hb = bf16_rn(a), bf16_rn(b)
    acc2 = np.float32(0.0)
    for u, v in zip(ha, hb):
        acc2 = np.float32(acc2 + np.float32(u * v))
    assert float(acc2) != float(np.dot(ha, hb))
