"""16-bit wire format of encoded symbols, written out plainly.

TEST INFRASTRUCTURE ONLY (tests, smoke check, benchmark CPU baseline).

Sec. II.B ("Design of the code on GF(65537)"): every element of F_65537 but
65536 fits in 16 bits, so an encoded symbol travels as 16 bits and the
positions that hold 65536 are announced separately (the paper puts them in
the header of each encoding packet).  Here a batch of encoded packets
``enc[rows][W]`` (values in [0, 65536]) becomes

* ``sym[rows][W]`` uint16, the symbol's low 16 bits (65536 -> 0), and
* ``esc[m][2]`` uint32, one ``(row, column)`` pair per symbol equal to 65536,
  sorted by row, then column (row = packet, column = codeword).

``from_wire`` inverts it.  Decoding from the wire format is ``from_wire`` of
the received packets followed by the ordinary decode.
"""
from __future__ import annotations

import numpy as np

ESCAPE = 65536


def to_wire(enc: np.ndarray):
    """(sym, esc) of encoded packets ``enc[rows][W]`` with values in [0, 65536]."""
    enc = np.asarray(enc)
    if enc.ndim != 2:
        raise ValueError("enc must be [rows][W]")
    if enc.size and int(enc.max()) > ESCAPE:
        raise ValueError("encoded symbols lie in [0, 65536]")
    sym = np.empty(enc.shape, dtype=np.uint16)
    esc = []
    for r in range(enc.shape[0]):
        for c in range(enc.shape[1]):
            v = int(enc[r, c])
            if v == ESCAPE:
                esc.append((r, c))
                sym[r, c] = 0
            else:
                sym[r, c] = v
    return sym, np.array(esc, dtype=np.uint32).reshape(-1, 2)


def from_wire(sym: np.ndarray, esc: np.ndarray) -> np.ndarray:
    """The encoded values ``[rows][W]`` uint32 back from (sym, esc)."""
    sym = np.asarray(sym)
    out = sym.astype(np.uint32)
    for r, c in np.asarray(esc, dtype=np.int64).reshape(-1, 2):
        if not (0 <= r < out.shape[0] and 0 <= c < out.shape[1]):
            raise ValueError(f"escape ({r}, {c}) outside the packets")
        if sym[r, c] != 0:
            raise ValueError(f"escaped symbol ({r}, {c}) is not sent as 0")
        out[r, c] = ESCAPE
    return out


def select_rows(esc: np.ndarray, rows) -> np.ndarray:
    """Escapes of the packets ``rows`` (in that order), renumbered to their index
    in ``rows``: what a receiver holding those packets stacked as rows 0.. sees."""
    esc = np.asarray(esc, dtype=np.uint32).reshape(-1, 2)
    out = []
    for i, r in enumerate(rows):
        for e in esc[esc[:, 0] == r]:
            out.append((i, int(e[1])))
    out.sort()
    return np.array(out, dtype=np.uint32).reshape(-1, 2)
