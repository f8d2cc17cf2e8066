"""Seeded synthetic inputs, shared by the tests, the benchmark and the CPU oracle runs.

This module holds no decoder arithmetic: it only draws the random numbers of the workload --
i.i.d. payload bits and unit-variance Gaussian noise -- from the counter-based generator
Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11), written here from that published definition.  Encoding, BPSK mapping and LLR scaling
are done by the consumers (the oracle on the CPU, the library's generator kernel on the GPU,
which implements the same Philox stream independently).

Counter layout (shared convention with the device generator):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (block, frame & 0xffffffff, stream, frame >> 32)
    stream 0: payload bits -- frame f, bit p uses word p // 32 = 4*block + lane, bit p % 32
    stream 1: noise        -- frame f, node j uses block j // 4; Box-Muller on (w0, w1) gives
              nodes 4b, 4b+1 and on (w2, w3) nodes 4b+2, 4b+3:
              U1 = ((w_even >> 8) + 1) / 2^24 in (0, 1],  U2 = (w_odd >> 8) / 2^24 in [0, 1),
              z_even = sqrt(-2 ln U1) cos(2 pi U2),  z_odd = sqrt(-2 ln U1) sin(2 pi U2).
"""
from __future__ import annotations

import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)

STREAM_PAYLOAD = 0
STREAM_NOISE = 1


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint32 counters (broadcast arrays), key bumped between rounds."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & _MASK for v in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    m0, m1 = np.uint64(PHILOX_M0), np.uint64(PHILOX_M1)
    for r in range(10):
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
    return tuple(v.astype(np.uint32) for v in (c0, c1, c2, c3))


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def philox_words(seed: int, stream: int, frame0: int, B: int, nblocks: int) -> np.ndarray:
    """uint32 [B][4*nblocks]: the raw stream of frames frame0 .. frame0+B-1."""
    k0, k1 = _key(seed)
    frames = np.arange(frame0, frame0 + B, dtype=np.uint64)[:, None]
    blocks = np.arange(nblocks, dtype=np.uint64)[None, :]
    f_lo = frames & _MASK
    f_hi = frames >> np.uint64(32)
    shape = (B, nblocks)
    w = philox4x32_10(np.broadcast_to(blocks, shape), np.broadcast_to(f_lo, shape),
                      np.full(shape, stream, np.uint64), np.broadcast_to(f_hi, shape), k0, k1)
    return np.stack(w, axis=-1).reshape(B, 4 * nblocks)


def payload_bits(seed: int, frame0: int, B: int, P: int) -> np.ndarray:
    """uint8 [B][P], one byte per bit, i.i.d. Bernoulli(1/2)."""
    nwords = (P + 31) // 32
    w = philox_words(seed, STREAM_PAYLOAD, frame0, B, (nwords + 3) // 4)[:, :nwords]
    bits = (w[:, :, None] >> np.arange(32, dtype=np.uint32)[None, None, :]) & np.uint32(1)
    return bits.reshape(B, nwords * 32)[:, :P].astype(np.uint8)


def unit_noise(seed: int, frame0: int, B: int, N: int) -> np.ndarray:
    """float64 [B][N] standard normal samples (Box-Muller on the Philox stream)."""
    nblocks = (N + 3) // 4
    w = philox_words(seed, STREAM_NOISE, frame0, B, nblocks).reshape(B, nblocks, 2, 2)
    even = w[..., 0].astype(np.float64)
    odd = w[..., 1].astype(np.float64)
    u1 = (np.floor(even / 256.0) + 1.0) / 16777216.0
    u2 = np.floor(odd / 256.0) / 16777216.0
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.stack([r * np.cos(2.0 * np.pi * u2), r * np.sin(2.0 * np.pi * u2)], axis=-1)
    return z.reshape(B, nblocks * 4)[:, :N]


def unit_noise_chunked(seed: int, frame0: int, B: int, N: int, chunk: int = 4096):
    """Yield (frame offset, noise block) pieces so large batches never hold all noise at once."""
    for off in range(0, B, chunk):
        b = min(chunk, B - off)
        yield off, unit_noise(seed, frame0 + off, b, N)
