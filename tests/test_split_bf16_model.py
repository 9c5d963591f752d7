"""Error bound of the split-BF16 model product used by the tensor-core dense kernel, emulated in
numpy: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the model M = KR A3' is formed as
hi*hi + hi*lo + lo*hi with exact products and FP32-or-better accumulation.  The dropped lo*lo
term and the two roundings leave a relative error near 2^-16, against ~2^-8 for one BF16
product, which is why the loss derivative y = df/dm stays close to FP32 accuracy."""
import numpy as np


def bf16(x):
    """Round float32 values to bfloat16 (nearest, ties to even), returned as float32."""
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def test_bf16_rounding_is_nearest_even():
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 3.0e-3], np.float32)
    got = bf16(x)
    assert got[0] == 1.0 and got[1] == 1.0                   # tie: rounds to the even mantissa
    assert got[2] == np.float32(1.0 + 4 * 2.0 ** -8)         # tie: rounds up to the even mantissa
    assert got[3] == -2.5
    assert abs(got[4] - 3.0e-3) <= 3.0e-3 * 2.0 ** -8


def test_split_model_error_is_near_2_to_the_minus_16():
    rng = np.random.default_rng(0)
    R = 64
    KR = rng.standard_normal((128, R)).astype(np.float32)
    A3 = rng.standard_normal((128, R)).astype(np.float32)
    exact = KR.astype(np.float64) @ A3.astype(np.float64).T
    kh, ah = bf16(KR), bf16(A3)
    kl, al = bf16(KR - kh), bf16(A3 - ah)
    f = lambda u, v: u.astype(np.float64) @ v.astype(np.float64).T
    split = f(kh, ah) + f(kh, al) + f(kl, ah)
    single = f(kh, ah)
    scale = np.abs(KR).astype(np.float64) @ np.abs(A3).astype(np.float64).T   # sum_j |kr_j a_j|
    err_split = np.max(np.abs(split - exact) / scale)
    err_single = np.max(np.abs(single - exact) / scale)
    assert err_split < 2.0 ** -14          # ~2^-16 typical, 2^-14 worst-case bound per term
    assert err_single > 2.0 ** -10         # one BF16 product is ~2^-8 off
    assert err_split < err_single / 64
