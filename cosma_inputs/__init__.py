"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This package holds no part of the matrix-multiplication method: it only turns
(seed, stream, element index) into a number.  Both sides of every parity check
draw their operands from it, so that the oracle and the GPU path see the same
matrices without either one depending on the other.

Generator: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC'11).  It is counter based, so any element of any matrix
can be produced on its own -- the oracle regenerates only the rows of A and the
columns of B it samples, while the device fills whole matrices.

Element (r, c) of a rows x cols matrix has logical index e = r*cols + c (the
leading dimension of the storage plays no role).  One Philox call per element:
    counter = (lo32(e), hi32(e), stream, 0),  key = (lo32(seed), hi32(seed))
gives four words w0..w3; the distributions use w0 and w1:

  uniform  f64:  r53 = (w1 << 21) | (w0 >> 11);    x = r53 * 2^-52 - 1   in [-1, 1)
           f32:  r24 = w0 >> 8;                    x = r24 * 2^-23 - 1   in [-1, 1)
           bf16: the f32 value rounded to nearest-even bf16
  integer        x = (w0 mod 17) - 8                (integers in [-8, 8])
  loguniform     |x| = (1 + (w1 >> 9) * 2^-23) * 2^e,  e = ((w0 >> 1) mod 54) - 27,
                 sign from bit 0 of w0              (|x| in [2^-27, 2^27) ~ [7.5e-9, 1.3e8])

Every value above is exact in its target type, so host and device agree bit for
bit.  The device half lives in csrc/philox_fill.cu.
"""

from .philox import (  # noqa: F401
    KINDS,
    philox4x32_10,
    matrix,
    entries,
    rows,
    cols,
    STREAM_A,
    STREAM_B,
    grouped_dims,
)
