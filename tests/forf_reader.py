"""An independent reader of the FOR1 bytes (frame-of-reference delta
bit-packing in blocks of 128 keys), written from the format's definition with
Python integers and numpy, sharing no code with the C reference in
``oracle/for_bp128.c`` or with the CUDA codec.  Used to pin both."""
from __future__ import annotations

import numpy as np


def _pad16(x: int) -> int:
    return (x + 15) & ~15


def parse(blob: bytes) -> dict:
    assert blob[:4] == b"FOR1", "magic"
    kb = int.from_bytes(blob[4:8], "little")
    n = int.from_bytes(blob[8:16], "little")
    B = int.from_bytes(blob[16:24], "little")
    W = int.from_bytes(blob[24:32], "little")
    assert kb in (4, 8) and B == -(-n // 128)
    ob = 32
    ow = ob + _pad16(kb * B)
    op = ow + _pad16(B)
    assert len(blob) == op + 4 * W, "length"
    dt = np.uint32 if kb == 4 else np.uint64
    base = np.frombuffer(blob, dtype=dt, count=B, offset=ob)
    width = np.frombuffer(blob, dtype=np.uint8, count=B, offset=ow)
    pay = blob[op:]
    pads = blob[ob + kb * B:ow] + blob[ow + B:op]
    return {"key_bytes": kb, "n": n, "blocks": B, "words": W, "base": base, "width": width, "payload": pay,
            "pads_zero": pads == bytes(len(pads))}


def decode(blob: bytes) -> np.ndarray:
    p = parse(blob)
    n, kb = p["n"], p["key_bytes"]
    out = np.empty(n, dtype=np.uint32 if kb == 4 else np.uint64)
    byte = 0
    mask64 = (1 << 64) - 1
    for b in range(p["blocks"]):
        w = int(p["width"][b])
        nbytes = 16 * w  # 4 w words
        bits = int.from_bytes(p["payload"][byte:byte + nbytes], "little")
        key = int(p["base"][b])
        for i in range(min(128, n - 128 * b)):
            g = (bits >> (i * w)) & ((1 << w) - 1)
            key = (key + g) & mask64
            out[128 * b + i] = key
        byte += nbytes
    assert byte == len(p["payload"]), "payload length"
    return out


def size(keys: np.ndarray) -> int:
    """The closed-form FOR1 length: header, bases, widths and 4 w_b words per
    block, w_b the bit length of the block's largest gap."""
    n, kb = keys.size, keys.itemsize
    B = -(-n // 128)
    k = keys.astype(object)
    W = 0
    for b in range(B):
        blk = k[128 * b:128 * b + 128]
        g = max((int(blk[i]) - int(blk[i - 1]) for i in range(1, len(blk))), default=0)
        W += 4 * g.bit_length()
    return 32 + _pad16(kb * B) + _pad16(B) + 4 * W
