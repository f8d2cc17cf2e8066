"""Seeded test inputs built on the CPU only: payload bits and noise from the input generator,
encoding, BPSK and LLR scaling by the oracle.  No input here ever comes from the CUDA path."""
import numpy as np

import oracle
from paper_1609_09358_gb300 import inputs


def oracle_code(N, K, crc_len, design_db=0.0, design_rate=None):
    return oracle.make_code(N, K, crc_len, design_db, design_rate)


def api_code(ocode):
    from paper_1609_09358_gb300 import api
    return api.PolarCode(ocode.N, ocode.K, ocode.crc_len, ocode.frozen.copy(), ocode.crc_poly)


def frames(ocode, ebn0_db, B, seed, frame0=0):
    """(payload uint8 [B][P] one byte per bit, llr float32 [B][N])."""
    pay = inputs.payload_bits(seed, frame0, B, ocode.P)
    x = oracle.encode_batch(pay, ocode)
    noise = inputs.unit_noise(seed, frame0, B, ocode.N)
    sigma = oracle.sigma_for(ebn0_db, ocode.P / ocode.N)
    return pay, oracle.channel_llr(x, noise, sigma)


def frames_large(ocode, ebn0_db, B, seed, chunk=8192):
    """Same as frames() for large B, generated in chunks."""
    pay = np.empty((B, ocode.P), np.uint8)
    llr = np.empty((B, ocode.N), np.float32)
    for off in range(0, B, chunk):
        b = min(chunk, B - off)
        p, l = frames(ocode, ebn0_db, b, seed, frame0=off)
        pay[off:off + b] = p
        llr[off:off + b] = l
    return pay, llr
