"""Second formulation of MTGP as F2 bit-matrices -- TEST INFRASTRUCTURE ONLY.

Every map of the recursion (Definition in Sec. 3.6) and of the tempering
(Definition in Sec. 3.7) is written as a 32x32 matrix over F2 built from what
the operation is -- a shift, a bit mask, a 4x32 matrix applied to the four
LSBs -- never by running the word operations of the C oracle on basis vectors.
The oracle's outputs are then compared with these matrix products (tests), and
the state-transition matrix F of Sec. 3.3 is assembled from the same blocks
for the period checks at reduced size.

Convention: a word is a column vector of its 32 bits, index 0 = the LSB, so
y = A x means bit b of y is the dot product of row b of A with the bits of x.
"""
from __future__ import annotations

import numpy as np

W = 32


def bits_of(word: int) -> np.ndarray:
    return np.array([(int(word) >> b) & 1 for b in range(W)], dtype=np.uint8)


def word_of(bits: np.ndarray) -> int:
    return int(sum(int(v & 1) << b for b, v in enumerate(bits)))


def eye() -> np.ndarray:
    return np.eye(W, dtype=np.uint8)


def shl(s: int) -> np.ndarray:
    """x << s: bit b of the result is bit b - s of x."""
    a = np.zeros((W, W), dtype=np.uint8)
    for b in range(s, W):
        a[b, b - s] = 1
    return a


def shr(s: int) -> np.ndarray:
    """x >> s (logical): bit b of the result is bit b + s of x."""
    a = np.zeros((W, W), dtype=np.uint8)
    for b in range(0, W - s):
        a[b, b + s] = 1
    return a


def diag_mask(mask: int) -> np.ndarray:
    return np.diag(bits_of(mask)).astype(np.uint8)


def low4_times(rows) -> np.ndarray:
    """u -> (four LSBs of u as a row vector) * Rows, Rows a 4x32 matrix.

    The four LSBs form a row vector whose leftmost component is the most
    significant of them (bit 3), so bit 3 of u selects row 0 and bit 0 selects
    row 3; the product is the XOR of the selected rows.
    """
    a = np.zeros((W, W), dtype=np.uint8)
    for j in range(4):
        a[:, 3 - j] = bits_of(rows[j])
    return a


def mm(*ms: np.ndarray) -> np.ndarray:
    out = ms[0].astype(np.int64)
    for m in ms[1:]:
        out = (out @ m.astype(np.int64)) & 1
    return out.astype(np.uint8)


def add(*ms: np.ndarray) -> np.ndarray:
    out = np.zeros_like(ms[0])
    for m in ms:
        out ^= m
    return out


def recursion_blocks(mask, sh1, sh2, R):
    """x_{N+i} = A0 x_i + A1 x_{1+i} + AM x_{M+i}  (Definition of Sec. 3.6).

    t = x_{1+i} + mask(x_i);  t = (I + SHL_sh1) t;  u = t + SHR_sh2 x_{M+i};
    x_{N+i} = (I + L_R) u, where L_R is u -> u_low4 * R.
    """
    fin = add(eye(), low4_times(R))
    t_map = add(eye(), shl(sh1))
    A0 = mm(fin, t_map, diag_mask(mask))
    A1 = mm(fin, t_map)
    AM = mm(fin, shr(sh2))
    return A0, A1, AM


def tempering_block(T):
    """o_{N+i} = x_{N+i} + H x_{M-1+i}  (Definition of Sec. 3.7).

    t = (I + SHR_16) y;  t = (I + SHR_8) t;  H y = t_low4 * T.
    """
    return mm(low4_times(T), add(eye(), shr(8)), add(eye(), shr(16)))


def simulate(mexp_N: int, pos: int, mask: int, sh1: int, sh2: int, R, T, state, n: int):
    """n uint32 outputs by matrix-vector products on the bit vectors of the words."""
    A0, A1, AM = recursion_blocks(mask, sh1, sh2, R)
    H = tempering_block(T)
    N, M = mexp_N, pos
    xs = [bits_of(w) for w in state]
    outs = []
    for k in range(n):
        xn = (mm(A0, xs[k][:, None]) ^ mm(A1, xs[k + 1][:, None]) ^ mm(AM, xs[k + M][:, None]))[:, 0]
        xs.append(xn)
        o = xn ^ mm(H, xs[M - 1 + k][:, None])[:, 0]
        outs.append(word_of(o))
    return np.array(outs, dtype=np.uint32), np.array([word_of(b) for b in xs[n:n + N]], dtype=np.uint32)


def transition_matrix(N: int, r: int, pos: int, mask: int, sh1: int, sh2: int, R) -> np.ndarray:
    """State transition F of Sec. 3.3 on the p = 32N - r effective bits.

    The full map acts on (x_0, ..., x_{N-1}) -> (x_1, ..., x_N); its state
    space drops the r LSBs of x_0, which the recursion never reads (x_0 enters
    only through the mask).  Coordinates of the p-dim space: the 32 - r MSBs of
    x_0 (bits r..31), then all bits of x_1, ..., x_{N-1}.
    """
    A0, A1, AM = recursion_blocks(mask, sh1, sh2, R)
    big = np.zeros((W * N, W * N), dtype=np.uint8)
    for i in range(N - 1):                         # new x_i = old x_{i+1}
        big[W * i:W * (i + 1), W * (i + 1):W * (i + 2)] = eye()
    last = slice(W * (N - 1), W * N)               # new x_{N-1} = x_N
    big[last, 0:W] ^= A0
    big[last, W:2 * W] ^= A1
    big[last, W * pos:W * (pos + 1)] ^= AM
    keep = [b for b in range(W * N) if b >= r]     # drop bits 0..r-1 of x_0
    return big[np.ix_(keep, keep)].copy()
