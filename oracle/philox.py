"""Counter-based normal draws of the filter: Philox4x32-10 plus Box-Muller.

The ETKF draws an initial ensemble (Sect. 2.2) and, with an AR(1) model driven
by noise (Sect. 2.1), a process-noise perturbation for every member at every
forecast.  Both implementations of the filter take those draws from the same
counter-based generator, each written from its published definition:

* Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw, "Parallel random
  numbers: as easy as 1, 2, 3", SC'11): multipliers 0xD2511F53 and 0xCD9E8D57,
  key increments 0x9E3779B9 and 0xBB67AE85.
* Box-Muller: u = (w + 0.5) / 2^32 for a 32-bit word w; a word pair (w_a, w_b)
  gives r = sqrt(-2 ln u_a), z0 = r cos(2 pi u_b), z1 = r sin(2 pi u_b).

Counter layout (shared definition): key = (seed mod 2^32, seed >> 32);
counter = (j // 4, member, frame, stream).  The four words of one call give the
normals with index 4(j//4) .. 4(j//4)+3: (w0, w1) -> the first pair, (w2, w3)
-> the second.  Streams: 0 = initial ensemble (frame 0: second block, frame 1:
first-block innovation), 1 = process noise of the forecast made at frame k.
"""

from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr: np.ndarray, key: np.ndarray) -> np.ndarray:
    """ctr: (..., 4) uint32, key: (..., 2) uint32 -> (..., 4) uint32 after 10 rounds."""
    c = [np.asarray(ctr[..., i], dtype=np.uint32).copy() for i in range(4)]
    k0 = np.asarray(key[..., 0], dtype=np.uint32).copy()
    k1 = np.asarray(key[..., 1], dtype=np.uint32).copy()
    with np.errstate(over="ignore"):
        for rnd in range(10):
            p0 = c[0].astype(np.uint64) * M0
            p1 = c[2].astype(np.uint64) * M1
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK).astype(np.uint32)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            if rnd < 9:
                k0 = k0 + W0
                k1 = k1 + W1
    return np.stack(c, axis=-1)


def box_muller(wa: np.ndarray, wb: np.ndarray):
    ua = (wa.astype(np.float64) + 0.5) / 4294967296.0
    ub = (wb.astype(np.float64) + 0.5) / 4294967296.0
    r = np.sqrt(-2.0 * np.log(ua))
    th = 2.0 * np.pi * ub
    return r * np.cos(th), r * np.sin(th)


def normals(seed: int, stream: int, frame: int, m: int, count: int) -> np.ndarray:
    """Standard normals Xi[j, i] for index j < count and member i < m (shape (count, m))."""
    nq = (count + 3) // 4
    q = np.arange(nq, dtype=np.uint32)
    mem = np.arange(m, dtype=np.uint32)
    Q, MEM = np.meshgrid(q, mem, indexing="ij")
    ctr = np.stack([Q, MEM, np.full_like(Q, np.uint32(frame & 0xFFFFFFFF)),
                    np.full_like(Q, np.uint32(stream & 0xFFFFFFFF))], axis=-1)
    key = np.empty(Q.shape + (2,), dtype=np.uint32)
    key[..., 0] = np.uint32(seed & 0xFFFFFFFF)
    key[..., 1] = np.uint32((seed >> 32) & 0xFFFFFFFF)
    w = philox4x32_10(ctr, key)
    z0, z1 = box_muller(w[..., 0], w[..., 1])
    z2, z3 = box_muller(w[..., 2], w[..., 3])
    z = np.stack([z0, z1, z2, z3], axis=1).reshape(4 * nq, m)
    return z[:count]
