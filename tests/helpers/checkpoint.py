"""The checkpoint byte layout of include/pt.h, written and read independently of the library
(test support): build a checkpoint from Python values, or decode one into the oracle's view."""
from __future__ import annotations

import struct

import numpy as np

MAGIC = b"PTCKPT02"


def fnv1a64(data: bytes) -> int:
    h = 1469598103934665603
    for b in data:
        h ^= b
        h = (h * 1099511628211) & 0xFFFFFFFFFFFFFFFF
    return h


def spins_to_words(spins_by_slot: np.ndarray) -> np.ndarray:
    """int8 [R][L][L] (+1 / -1, by slot) -> uint32 [W][2][L][L/2] bit planes."""
    R, L, _ = spins_by_slot.shape
    W = (R + 31) // 32
    words = np.zeros((W, 2, L, L // 2), np.uint64)
    for r in range(R):
        w, b = divmod(r, 32)
        up = (spins_by_slot[r] > 0).astype(np.uint64)
        for y in range(L):
            for c in range(2):
                x = 2 * np.arange(L // 2) + ((y + c) & 1)
                words[w, c, y] |= up[y, x] << np.uint64(b)
    return words.astype(np.uint32)


def words_to_spins(words: np.ndarray, R: int) -> np.ndarray:
    W, _, L, half = words.shape
    out = np.empty((R, L, L), np.int8)
    for r in range(R):
        w, b = divmod(r, 32)
        for y in range(L):
            for c in range(2):
                x = 2 * np.arange(half) + ((y + c) & 1)
                out[r, y, x] = np.where((words[w, c, y] >> b) & 1, 1, -1)
    return out


def build(L, betas, J, h, seed, t, e, rule, slot_of_temp, attempted, accepted, words,
          it=0) -> bytes:
    R = len(betas)
    head = MAGIC + struct.pack("<IIddQQQiiQ", L, R, J, h, seed, t, e, rule, 0, it)
    body = (np.asarray(betas, "<f8").tobytes() + np.asarray(slot_of_temp, "<i4").tobytes() +
            np.asarray(attempted, "<u8").tobytes() + np.asarray(accepted, "<u8").tobytes() +
            np.ascontiguousarray(words, "<u4").tobytes())
    data = head + body
    return data + struct.pack("<Q", fnv1a64(data))


def parse(data: bytes) -> dict:
    assert data[:8] == MAGIC
    L, R = struct.unpack_from("<II", data, 8)
    J, h = struct.unpack_from("<dd", data, 16)
    seed, t, e = struct.unpack_from("<QQQ", data, 32)
    rule, _ = struct.unpack_from("<ii", data, 56)
    it, = struct.unpack_from("<Q", data, 64)
    off = 72
    betas = np.frombuffer(data, "<f8", R, off); off += 8 * R
    sot = np.frombuffer(data, "<i4", R, off); off += 4 * R
    P = max(R - 1, 0)
    att = np.frombuffer(data, "<u8", P, off); off += 8 * P
    acc = np.frombuffer(data, "<u8", P, off); off += 8 * P
    W = (R + 31) // 32
    words = np.frombuffer(data, "<u4", W * 2 * L * (L // 2), off).reshape(W, 2, L, L // 2)
    off += 4 * words.size
    checksum, = struct.unpack_from("<Q", data, off)
    assert off + 8 == len(data) and checksum == fnv1a64(data[:off])
    return dict(L=L, R=R, J=J, h=h, seed=seed, t=t, e=e, rule=rule, it=it, betas=betas,
                slot_of_temp=sot, attempted=att, accepted=acc, words=words)
