"""The matrix partitioner of Section IV, read literally (oracle; test infrastructure only).

Section IV: the partitioner cuts A (M x K) into h horizontal slices of equal
size, B (K x N) into w vertical slices of equal size and C into the h x w
blocks between them, choosing h and w so that everything needed to update two
C blocks that share a block column is resident in the device memory dMemSize
at the same time (sizes counted in elements).

Reading (the paper gives the constraint, not the search):
  * two C blocks of one column (rows i and i+1 of column j) need two A slices,
    the single B slice of the column and the two C blocks:
        2 * (M/h) * K + K * (N/w) + 2 * (M/h) * (N/w) <= dMemSize;
  * equal sizes: h divides M and w divides N;
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
