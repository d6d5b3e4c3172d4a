"""The componentwise bounds the GPU parity tests use (tests/bounds.py) checked on the CPU.

The Ozaki form is emulated exactly here, from its definition: each operand row (column of B)
is scaled by the power of two above its largest entry, its fixed-point value is truncated to S
digits of 6 bits, and the digit products with s + t <= S + 1 are summed in exact integer
arithmetic (Python integers).  The only error left is the method's own (truncation and dropped
products), so the emulation must sit inside the bound without its slack factor; and a result
with one plausible mistake (a dropped digit product, a wrong weight, one wrong element) must
break the bound, so the bound is tight enough to catch it.
"""
from fractions import Fraction

import numpy as np
import pytest

import synth
from bounds import SLACK, bf16x3_bound, ozaki_bound, worst_ratio

BETA = 6


def _digits(v, e, S):
    """the S signed 6-bit digits of v * 2^-e (|v| < 2^e), truncated, most significant first"""
    F = int(Fraction(abs(v)) * 2 ** (S * BETA - e))   # floor of the exact fixed-point value
    d = [(F >> (BETA * (S - s))) & 63 for s in range(1, S + 1)]
    return [-x for x in d] if v < 0 else d


def _exp(row):
    m = float(np.abs(row).max())
    return int(np.frexp(m)[1]) if m > 0 else 0


def ozaki_emulate(A, B, S, drop=None, weight_shift=None):
    M, K = A.shape
    N = B.shape[1]
    ea = [_exp(A[i]) for i in range(M)]
    fb = [_exp(B[:, j]) for j in range(N)]
    da = [[_digits(A[i, k], ea[i], S) for k in range(K)] for i in range(M)]
    db = [[_digits(B[k, j], fb[j], S) for j in range(N)] for k in range(K)]
    C = np.zeros((M, N))
    for i in range(M):
        for j in range(N):
            acc = Fraction(0)
            for s in range(1, S + 1):
                for t in range(1, S + 2 - s):
                    if drop == (s, t):
                        continue
                    w = BETA * (s + t) + (1 if weight_shift == (s, t) else 0)
                    p = sum(da[i][k][s - 1] * db[k][j][t - 1] for k in range(K))
                    acc += Fraction(p, 2 ** w)
            C[i, j] = float(acc * Fraction(2) ** (ea[i] + fb[j]))
    return C


def _inputs(seed, M, K, N):
    A = synth.matrix(M, K, seed, 0, synth.LOGSPREAD)
    B = synth.matrix(K, N, seed, 1, synth.LOGSPREAD)
    exact = np.array([[float(sum(Fraction(A[i, k]) * Fraction(B[k, j]) for k in range(K))) for j in range(N)]
                      for i in range(M)])
    return A, B, exact


@pytest.mark.parametrize("S", [8, 9])
def test_ozaki_emulation_inside_bound(S):
    A, B, exact = _inputs(501 + S, 6, 40, 5)
    got = ozaki_emulate(A, B, S)
    bound = ozaki_bound(A, B, 1.0, 0.0, None, S) / SLACK
    assert worst_ratio(got, exact, bound) <= 1.0


@pytest.mark.parametrize("mistake", ["drop", "weight", "entry"])
def test_ozaki_bound_catches_mistakes(mistake):
    S = 8
    A, B, exact = _inputs(601, 6, 40, 5)
    if mistake == "drop":        # one leading digit product left out
        got = ozaki_emulate(A, B, S, drop=(1, 2))
    elif mistake == "weight":    # one product added with half its weight
        got = ozaki_emulate(A, B, S, weight_shift=(3, 4))
    else:                        # one element off by 1e-7 of its row / column scale 2^(e_i + f_j)
        got = ozaki_emulate(A, B, S)
        got[2, 3] += 1e-7 * 2.0 ** (_exp(A[2]) + _exp(B[:, 3]))
    bound = ozaki_bound(A, B, 1.0, 0.0, None, S)
    assert worst_ratio(got, exact, bound) > 1.0


def _bf16(x):
    """round-to-nearest-even FP32 -> bf16 (as FP32), from the bit pattern"""
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def test_bf16x3_split_inside_bound():
    """The BF16x3 split and its six products, in FP64 (no tensor-core accumulation): inside the
    split share of the bound; dropping one of the two 2^-8 products breaks the whole bound."""
    rng = np.random.default_rng(7)
    A = rng.uniform(-1, 1, (20, 300)).astype(np.float32)
    B = rng.uniform(-1, 1, (300, 16)).astype(np.float32)

    def pieces(x):
        h = _bf16(x)
        r1 = (x - h).astype(np.float32)
        m = _bf16(r1)
        r2 = (r1 - m).astype(np.float32)
        return [p.astype(np.float64) for p in (h, m, _bf16(r2))]

    ha, ma, la = pieces(A)
    hb, mb, lb = pieces(B)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    six = ha @ hb + ha @ mb + ma @ hb + ha @ lb + ma @ mb + la @ hb
    AB = np.abs(A.astype(np.float64)) @ np.abs(B.astype(np.float64))
    assert worst_ratio(six, exact, 2.0 ** -25 * AB) <= 1.0
    bound = bf16x3_bound(A, B, 1.0, 0.0, None)
    assert worst_ratio(six - ha @ mb, exact, bound) > 1.0


def _rz32(x):
    """float64 values rounded toward zero to FP32 (the tensor cores' accumulator rounding)"""
    x = np.asarray(x, dtype=np.float64)
    r = x.astype(np.float32)
    over = np.abs(r.astype(np.float64)) > np.abs(x)
    r[over] = np.nextafter(r[over], np.float32(0))
    return r


def _pieces(x):
    h = _bf16(x)
    r1 = (x - h).astype(np.float32)
    m = _bf16(r1)
    r2 = (r1 - m).astype(np.float32)
    return [p.astype(np.float64) for p in (h, m, _bf16(r2))]


def bf16x3_emulate(A, B, drain, small_k=2048):
    """The BF16x3 form's accumulation: every 16-long K step of a piece product is summed exactly
    (one MMA) and added into an FP32 accumulator that rounds toward zero; hh has its own
    accumulator, emptied into an exact sum every `drain` of K, and the five small products share
    one emptied every `small_k` of K."""
    ha, ma, la = _pieces(A)
    hb, mb, lb = _pieces(B)
    small = [(ha, mb), (ma, hb), (ha, lb), (ma, mb), (la, hb)]
    K = A.shape[1]
    total = np.zeros((A.shape[0], B.shape[1]))
    acc_h = np.zeros_like(total, dtype=np.float32)
    acc_s = np.zeros_like(total, dtype=np.float32)
    for k0 in range(0, K, 16):
        k1 = min(K, k0 + 16)
        acc_h = _rz32(acc_h.astype(np.float64) + ha[:, k0:k1] @ hb[k0:k1])
        acc_s = _rz32(acc_s.astype(np.float64) + sum(a[:, k0:k1] @ b[k0:k1] for a, b in small))
        if k1 % drain == 0 or k1 == K:
            total += acc_h
            acc_h[:] = 0
        if k1 % small_k == 0 or k1 == K:
            total += acc_s
            acc_s[:] = 0
    return total


@pytest.mark.parametrize("drain", [128, 512])
def test_bf16x3_accumulation_inside_bound(drain):
    """Round-toward-zero accumulation with drains every `drain` of K sits inside the bound for
    that drain length without its slack; positive inputs make every rounding error point the
    same way (the worst case for a truncating accumulator)."""
    rng = np.random.default_rng(11)
    A = rng.uniform(0, 1, (6, 4096)).astype(np.float32)
    B = rng.uniform(0, 1, (4096, 5)).astype(np.float32)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    got = bf16x3_emulate(A, B, drain)
    assert worst_ratio(got, exact, bf16x3_bound(A, B, 1.0, 0.0, None, drain=drain) / SLACK) <= 1.0


def test_bf16x3_bound_catches_an_undrained_accumulator():
    """Without the periodic drains (one accumulator over the whole K = 16384, 1024 truncating
    additions) the error leaves the bound for drains every 512 of K."""
    rng = np.random.default_rng(12)
    A = rng.uniform(0, 1, (6, 16384)).astype(np.float32)
    B = rng.uniform(0, 1, (16384, 5)).astype(np.float32)
    exact = A.astype(np.float64) @ B.astype(np.float64)
    got = bf16x3_emulate(A, B, drain=16384, small_k=16384)
    assert worst_ratio(got, exact, bf16x3_bound(A, B, 1.0, 0.0, None, drain=512)) > 1.0
