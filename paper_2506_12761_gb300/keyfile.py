"""Cloud-key files: save and reload the evaluation key (BK, KSK) of the
paper's parameter set so that a server can restart without a new key.

Format (little-endian): magic b"VLPRKEY1", seven int32 parameters
(n, N, k, l, bg_bits, ks_t, ks_base_bits), two uint64 word counts, the
SHA-256 of the payload, then the BK words and the KSK words in the layouts
velopir_load_cloud_key takes.  Loading checks the magic, the parameters, the
sizes and the digest and raises ValueError on any mismatch.
"""
from __future__ import annotations

import hashlib
import struct

import numpy as np

MAGIC = b"VLPRKEY1"
PARAMS = (630, 1024, 1, 3, 7, 8, 2)
BK_WORDS = 630 * 6 * 2 * 1024
KSK_WORDS = 1024 * 8 * 4 * 631
_HDR = struct.Struct("<8s7i2Q32s")


def save_cloud_key(path: str, bk: np.ndarray, ksk: np.ndarray) -> None:
    bk = np.ascontiguousarray(bk, dtype=np.uint32).reshape(-1)
    ksk = np.ascontiguousarray(ksk, dtype=np.uint32).reshape(-1)
    if bk.size != BK_WORDS or ksk.size != KSK_WORDS:
        raise ValueError("cloud key arrays have the wrong size for the paper's parameter set")
    h = hashlib.sha256()
    h.update(bk.astype("<u4").tobytes())
    h.update(ksk.astype("<u4").tobytes())
    with open(path, "wb") as f:
        f.write(_HDR.pack(MAGIC, *PARAMS, bk.size, ksk.size, h.digest()))
        f.write(bk.astype("<u4").tobytes())
        f.write(ksk.astype("<u4").tobytes())


def load_cloud_key(path: str) -> tuple[np.ndarray, np.ndarray]:
    with open(path, "rb") as f:
        head = f.read(_HDR.size)
        if len(head) != _HDR.size:
            raise ValueError("truncated cloud-key file")
        magic, *rest = _HDR.unpack(head)
        params, nbk, nksk, digest = tuple(rest[:7]), rest[7], rest[8], rest[9]
        if magic != MAGIC:
            raise ValueError("not a cloud-key file")
        if params != PARAMS or nbk != BK_WORDS or nksk != KSK_WORDS:
            raise ValueError(f"cloud-key file is for parameters {params}, sizes {nbk}/{nksk}")
        bk = np.frombuffer(f.read(4 * nbk), dtype="<u4")
        ksk = np.frombuffer(f.read(4 * nksk), dtype="<u4")
    if bk.size != nbk or ksk.size != nksk:
        raise ValueError("truncated cloud-key file")
    h = hashlib.sha256()
    h.update(bk.tobytes())
    h.update(ksk.tobytes())
    if h.digest() != digest:
        raise ValueError("cloud-key file is corrupt (digest mismatch)")
    return bk.astype(np.uint32), ksk.astype(np.uint32)
