"""Componentwise error bounds of the two tensor-core forms, derived from their arithmetic.

Each bound is an upper bound on |C_gpu[i, j] - C[i, j]| for every element, where C is the
exact product of the (FP64, or FP32 widened to FP64) inputs, so the GPU result can be checked
element by element against the oracle: a wrong small entry fails even when the relative
Frobenius norm, dominated by the largest entries, would hide it.  The oracle's own FP64
rounding (k ascending) is added to each bound.

Ozaki form (S digits of beta bits per operand row / column, truncated; digit products with
s + t <= S + 1 kept, each summed exactly in FP32 over K chunks of at most 4096, FP64
accumulation).  With x_k = a_ik 2^-e_i and y_k = b_kj 2^-f_j (|x|, |y| < 1 after the
power-of-two row / column scaling), per k:
    |x y - computed| <= 2^(-beta S) (|x_k| + |y_k|)          truncation of each operand
                        + D_S                                 dropped products s + t >= S + 2
    D_S = sum_{m=S+2}^{2S} (2S + 1 - m) (2^beta - 1)^2 2^(-beta m)
so, summed over k and scaled back,
    |err_ij| <= |alpha| [2^(-beta S) (2^e_i ||b_j||_1 + 2^f_j ||a_i||_1) + K D_S 2^(e_i + f_j)
                         + n_add 2^-53 (|A||B|)_ij] + kc 2^-52 (|alpha| (|A||B|)_ij + |beta| |C0_ij|)
with n_add the FP64 additions of weighted exact partial sums per element and kc the pipeline's
K chunks (each rounds once more into C).  The K D_S 2^(e+f) term is this design's accuracy
scale: relative to each row's and column's largest entry, not to (|A||B|)_ij, because the
digits are cut from the row's fixed-point value.

BF16x3 form (x = h + m + l, each the bf16 rounding of what is left; products hh, hm, mh, hl,
mm, lh; the leading product hh in its own FP32 tensor-core accumulator drained every L of K
(L = 512) into double-float registers, the five small products in a second accumulator drained
every 2048 of K):
    splitting and dropped products (ml, lm, ll):   <= 2^-25 |x| |y| per k
    hh accumulation inside one L-long chunk:        L / 16 MMA additions, each rounding toward
                                                    zero by at most one ulp (2^-23) of the running
                                                    sum, <= (L / 16) 2^-23 |x| |y|, plus the MMA's
                                                    own 16-term sum, <= 2^-20 |x| |y|
    small products inside one 2048-long stretch:    640 additions to a sum below 2^-7 of
                                                    sum |x| |y|: <= 2^-20 |x| |y|
    together (the accumulation term below):         ((L / 16) 2^-23 + 2^-19) |x| |y|
    the result rounded to FP32 (once per K chunk):  kc 2^-24 (|alpha| (|A||B|)_ij + |beta| |C0_ij|)
"""
import math

import numpy as np

OZAKI_BETA = 6
OZAKI_EXACT_CHUNK = 4096
SLACK = 2.0


def _exps(rowmax):
    """e with max < 2^e per row (frexp: max = m 2^e, m in [0.5, 1)); 0 for an all-zero row."""
    _, e = np.frexp(rowmax)
    return np.where(rowmax > 0, e, 0).astype(np.float64)


def ozaki_bound(Aop, Bop, alpha, beta, C0, S, kchunks=1):
    """Elementwise bound for op(A) (M x K) times op(B) (K x N) in the Ozaki form with S digits."""
    Aop = np.asarray(Aop, dtype=np.float64)
    Bop = np.asarray(Bop, dtype=np.float64)
    K = Aop.shape[1]
    b = OZAKI_BETA
    absA, absB = np.abs(Aop), np.abs(Bop)
    e = _exps(absA.max(axis=1) if K else np.zeros(Aop.shape[0]))
    f = _exps(absB.max(axis=0) if K else np.zeros(Bop.shape[1]))
    AB = absA @ absB
    D = sum((2 * S + 1 - m) * (2.0 ** b - 1) ** 2 * 2.0 ** (-b * m) for m in range(S + 2, 2 * S + 1))
    products = S * (S + 1) // 2
    n_add = products * max(1, math.ceil(K / OZAKI_EXACT_CHUNK)) + 2
    trunc = 2.0 ** (-b * S) * (np.exp2(e)[:, None] * absB.sum(axis=0)[None, :] +
                               absA.sum(axis=1)[:, None] * np.exp2(f)[None, :])
    dropped = K * D * np.exp2(e[:, None] + f[None, :])
    acc = n_add * 2.0 ** -53 * AB
    cterm = 0.0 if C0 is None or beta == 0 else abs(beta) * np.abs(C0)
    out = kchunks * 2.0 ** -52 * (abs(alpha) * AB + cterm)
    oracle_rounding = (K + 2) * 2.0 ** -53 * (abs(alpha) * AB + cterm)
    return SLACK * (abs(alpha) * (trunc + dropped + acc) + out + oracle_rounding)


BF16X3_DRAIN = 512


def bf16x3_bound(Aop, Bop, alpha, beta, C0, kchunks=1, drain=BF16X3_DRAIN):
    """Elementwise bound for FP32 op(A) times op(B) in the BF16x3 form (result rounded to FP32),
    the leading product's accumulator drained every `drain` of K."""
    Aop = np.asarray(Aop, dtype=np.float64)
    Bop = np.asarray(Bop, dtype=np.float64)
    K = Aop.shape[1]
    AB = np.abs(Aop) @ np.abs(Bop)
    cterm = 0.0 if C0 is None or beta == 0 else abs(beta) * np.abs(C0)
    split = 2.0 ** -25 * AB
    accum = ((drain / 16) * 2.0 ** -23 + 2.0 ** -19) * AB
    out = (kchunks + 1) * 2.0 ** -24 * (abs(alpha) * AB + cterm)
    oracle_rounding = (K + 2) * 2.0 ** -53 * (abs(alpha) * AB + cterm)
    return SLACK * (abs(alpha) * (split + accum) + out + oracle_rounding)


def op(x, t):
    """op(X) for a stored operand: X itself for 'N', its transpose for 'T'."""
    x = np.asarray(x, dtype=np.float64)
    return x if t == "N" else x.T


def worst_ratio(got, ref, bound):
    """max over elements of |got - ref| / bound (<= 1 passes); NaN anywhere fails."""
    err = np.abs(np.asarray(got, dtype=np.float64) - np.asarray(ref, dtype=np.float64))
    if not np.isfinite(err).all():
        return float("inf")
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bound > 0, err / bound, np.where(err > 0, np.inf, 0.0))
    return float(r.max()) if r.size else 0.0
