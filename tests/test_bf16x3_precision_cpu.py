"""The precision scheme of the tensor-core contraction, emulated on the CPU: each
operand value is split v = hi + lo with hi = bf16(v) and lo = bf16(v - hi) (round to
nearest even), and the product is hi_A hi_B + hi_A lo_B + lo_A hi_B with FP32
accumulation (BF16 x BF16 products are exact in FP32).  On the field contraction of
Eq. 2 (Sec. 2.1) for random spins the result stays within the 1e-5 normwise bound the
FP32 paths are held to, while a single BF16 product misses it by two orders."""
import numpy as np

from oracle import oracle as orc
from paper_1211_6234_b300 import inputs


def bf16(x):
    """Round FP32 values to BF16 (nearest, ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return r.astype(np.uint32).view(np.float32)


def split(x):
    x = np.asarray(x, np.float32)
    hi = bf16(x)
    return hi, bf16(x - hi)


def test_bf16_rounding_is_nearest_even():
    one = np.float32(1.0)
    eps = np.float32(2.0 ** -7)                                   # spacing of bf16 in [1, 2)
    assert bf16(np.array([one + eps / 2]))[0] == one              # a tie goes to the even neighbour
    assert bf16(np.array([one + 3 * eps / 2]))[0] == one + 2 * eps
    assert bf16(np.array([one + eps / 2 + np.float32(2.0 ** -20)]))[0] == one + eps   # above the tie
    x = np.random.default_rng(1).normal(size=10000).astype(np.float32)
    hi, lo = split(x)
    assert np.all(np.abs(x - hi) <= 2.0 ** -8 * np.abs(x))        # half a spacing of 8 bits
    assert np.all(np.abs(x - hi - lo) <= 2.0 ** -16 * np.abs(x))  # 16 bits kept by the pair


def test_split_bf16x3_contraction_meets_the_field_bound():
    L, R = 16, 8
    N = L * L
    W = orc.wtilde(L, 16, True)
    s = inputs.random_spins(L, R, seed=21)
    # rows: (output component b, site q); columns: (input component a, source m) -- Eq. 2
    A = np.zeros((3 * N, 3 * N))
    y, x = np.divmod(np.arange(N), L)
    dy = (y[:, None] - y[None, :]) % L
    dx = (x[:, None] - x[None, :]) % L
    blk = {(0, 0): 0, (0, 1): 1, (1, 0): 1, (1, 1): 2, (2, 2): 3}
    for (b, a), c in blk.items():
        A[b * N:(b + 1) * N, a * N:(a + 1) * N] = W[c][dy, dx]
    B = s.reshape(R, 3 * N).T                                     # [3N][R]
    D64 = A @ B
    assert np.allclose(D64.T.reshape(R, 3, L, L)[0], orc.field(W, s[0]), atol=1e-12)
    Ah, Al = split(A)
    Bh, Bl = split(B)
    D3 = (Ah @ Bh).astype(np.float32) + (Ah @ Bl).astype(np.float32) + (Al @ Bh).astype(np.float32)
    D1 = Ah @ Bh
    err3 = np.abs(D3 - D64).max() / np.abs(D64).max()
    err1 = np.abs(D1 - D64).max() / np.abs(D64).max()
    assert err3 < 1e-5, err3
    assert err1 > 1e-4, err1                                      # one product is not enough
