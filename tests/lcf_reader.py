"""Independent reader of the "LCF1" byte format, for the tests only.

It parses a blob with ``struct``/numpy and recomputes, with Python integers,
what the paper fixes about it:

* Def. 1: Dec(K^c)[i] = K[i] -- ``reconstruct`` rebuilds every key from the
  segments and the residuals read bit by bit;
* Def. 2: |Delta[i]| <= eps for every residual;
* Sec. II-A: ceil(log2(2 eps + 1)) bits per residual bound every width, and the
  size of K^c is the model bytes plus the residual bits (``closed_form_size``).

It shares no code with ``oracle/`` or with the CUDA library.
"""
from __future__ import annotations

import struct

import numpy as np

HEADER = struct.Struct("<4sHHIIQQQQQQ")


def _pad16(x: int) -> int:
    return (x + 15) // 16 * 16


def layout(kb: int, C: int, L: int, W: int, NL: int, list_mode: bool):
    """Byte offsets of every array and the total size of a blob."""
    names, sizes = [], []
    if list_mode:
        names += ["list_key_begin", "list_chunk_begin", "list_eps", "list_chunk_log2"]
        sizes += [8 * (NL + 1), 8 * (NL + 1), 8 * NL, NL]
    names += ["chunk_key_begin", "chunk_seg_begin", "chunk_word_begin", "seg_icpt", "seg_slope",
              "seg_bitoff", "seg_start", "seg_width", "payload"]
    sizes += [8 * (C + 1)] * 3 + [kb * L, 8 * L, 4 * L, 2 * L, L, 8 * W]
    off, offs = 64, {}
    for nm, sz in zip(names, sizes):
        offs[nm] = (off, sz)
        off += _pad16(sz)
    return offs, off


def parse(blob: bytes) -> dict:
    magic, ver, flags, kb, log2, N, eps, C, L, W, NL = HEADER.unpack_from(blob, 0)
    assert magic == b"LCF1" and ver == 1
    list_mode = bool(flags & 1)
    offs, total = layout(kb, C, L, W, NL, list_mode)
    assert total == len(blob), (total, len(blob))
    kdt = np.dtype("<u4") if kb == 4 else np.dtype("<u8")
    dts = {"list_key_begin": "<u8", "list_chunk_begin": "<u8", "list_eps": "<u8",
           "list_chunk_log2": "u1", "chunk_key_begin": "<u8", "chunk_seg_begin": "<u8",
           "chunk_word_begin": "<u8", "seg_icpt": kdt, "seg_slope": "<i8", "seg_bitoff": "<u4",
           "seg_start": "<u2", "seg_width": "u1", "payload": "<u8"}
    out = {"key_bytes": kb, "chunk_log2": log2, "n": N, "eps": eps, "chunks": C, "segments": L,
           "words": W, "lists": NL, "list_mode": list_mode}
    for nm, (o, sz) in offs.items():
        out[nm] = np.frombuffer(blob, dtype=dts[nm], count=sz // np.dtype(dts[nm]).itemsize,
                                offset=o)
    return out


def segments(p: dict):
    """Per segment: (chunk, absolute start, length)."""
    ckb, csb = p["chunk_key_begin"], p["chunk_seg_begin"]
    st = p["seg_start"].astype(np.int64)
    res = []
    for c in range(p["chunks"]):
        a, b = int(csb[c]), int(csb[c + 1])
        n_c = int(ckb[c + 1] - ckb[c])
        for j in range(a, b):
            e = int(st[j + 1]) if j + 1 < b else n_c
            res.append((c, int(ckb[c]) + int(st[j]), e - int(st[j])))
    return res


def _bits(payload: np.ndarray, pos: int, w: int) -> int:
    v = 0
    for b in range(w):
        p = pos + b
        v |= ((int(payload[p >> 6]) >> (p & 63)) & 1) << b
    return v


def residuals(p: dict):
    """Every stored residual Delta (zigzag decoded), per segment, as Python ints."""
    pay, cwb = p["payload"], p["chunk_word_begin"]
    out = []
    for j, (c, s, n) in enumerate(segments(p)):
        w = int(p["seg_width"][j])
        base = 64 * int(cwb[c]) + int(p["seg_bitoff"][j])
        r = [0]
        for t in range(1, n):
            z = _bits(pay, base + w * (t - 1), w)
            r.append(-(z >> 1) - 1 if z & 1 else z >> 1)
        out.append(r)
    return out


def reconstruct(p: dict) -> list:
    """Dec(K^c) from the segments and residuals, in exact Python integers:
    K[s_j + t] = icpt_j + floor(M_j t / 2^32) + Delta."""
    keys = []
    res = residuals(p)
    for j, (c, s, n) in enumerate(segments(p)):
        icpt = int(p["seg_icpt"][j])
        M = int(p["seg_slope"][j])
        for t in range(n):
            keys.append(icpt + ((M * t) >> 32) + res[j][t])
    return keys


def predictions(p: dict) -> list:
    """floor(f(i)) of every key from the segments alone, in exact Python
    integers reduced to the key width: icpt_j + floor(M_j t / 2^32)."""
    mod = 1 << (8 * p["key_bytes"])
    out = []
    for j, (c, s, n) in enumerate(segments(p)):
        icpt = int(p["seg_icpt"][j])
        M = int(p["seg_slope"][j])
        out.extend((icpt + ((M * t) >> 32)) % mod for t in range(n))
    return out


def closed_form_size(p: dict) -> int:
    """Sec. II-A size(K^c) = size(f) + residual bits, restated for this format:
    header + chunk directory + per-segment model + packed residual words, with W
    the sum over chunks of the even-rounded ceil(sum_j w_j (n_j - 1) / 64)."""
    W = 0
    segs = segments(p)
    per_chunk = {}
    for j, (c, s, n) in enumerate(segs):
        per_chunk[c] = per_chunk.get(c, 0) + int(p["seg_width"][j]) * (n - 1)
    for c in range(p["chunks"]):
        words = -(-per_chunk.get(c, 0) // 64)
        W += words + (words & 1)
    assert W == p["words"]
    _, total = layout(p["key_bytes"], p["chunks"], len(segs), W, p["lists"], p["list_mode"])
    return total
