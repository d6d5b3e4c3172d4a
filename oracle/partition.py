"""The matrix partitioner of Section IV, read literally (oracle; test infrastructure only).

Section IV: hclMatrixPartitioner splits A (M x K) into h equal horizontal
slices, B (K x N) into w equal vertical slices and C into h x w equal blocks,
so that the data needed to update any two blocks of C in the same column fits
in the device memory dMemSize (counted in elements).

Reading (the paper states the constraint, not the search):
  * "two blocks of C in the same column" (i and i+1 of column j) need two A
    slices, the one B slice of that column and two C blocks:
        2 * (M/h) * K + K * (N/w) + 2 * (M/h) * (N/w) <= dMemSize;
  * "equal" slices: h divides M and w divides N;
  * among the (h, w) that fit, the fewest blocks h * w; ties go to the smaller
    footprint, then to the larger h.
The worked example of Section IV (A 4 x 8, B 8 x 4, C 4 x 4, 44 elements,
Fig. 2 caption: 4 slices of A, 2 of B, 8 blocks of C) gives (h, w) = (4, 2).
"""


def footprint(M, N, K, h, w):
    """Elements resident for two C blocks of one column (two A slices, one B slice, two C blocks)."""
    mb, nb = M // h, N // w
    return 2 * mb * K + K * nb + 2 * mb * nb


def partition(M, N, K, dmem_elems):
    """(h, w) per the reading above, or None when no equal split fits."""
    best = None
    for h in range(1, M + 1):
        if M % h:
            continue
        for w in range(1, N + 1):
            if N % w:
                continue
            f = footprint(M, N, K, h, w)
            if f > dmem_elems:
                continue
            key = (h * w, f, -h)
            if best is None or key < best[0]:
                best = (key, (h, w))
    return None if best is None else best[1]
