"""Decoding of the column-packed code layout of include/qiht.h (test helper).

Pure data layout, no arithmetic of the method: word q of column j holds rows
q*G .. q*G+G-1 (G = 32/bits); the code of row q*G + 4k + p sits at bit
8p + bits*k."""
import numpy as np


def ld_words(rows: int, bits: int) -> int:
    G = 32 // bits
    w = (rows + G - 1) // G
    return (w + 3) & ~3


def unpack(words: np.ndarray, rows: int, cols: int, bits: int) -> np.ndarray:
    """words (cols * ld_words u32) -> codes (rows x cols, uint16)."""
    G = 32 // bits
    ldw = ld_words(rows, bits)
    w = np.asarray(words).view(np.uint32).reshape(cols, ldw)
    r = np.arange(rows)
    wi, k = r // G, r % G
    shift = (8 * (k % 4) + bits * (k // 4)).astype(np.uint32)
    return ((w[:, wi] >> shift[None, :]) & np.uint32((1 << bits) - 1)).T.astype(np.uint16)


def padding_is_zero(words: np.ndarray, rows: int, cols: int, bits: int) -> bool:
    """Codes of rows past `rows` (up to the column's padded length) are 0."""
    G = 32 // bits
    ldw = ld_words(rows, bits)
    w = np.asarray(words).view(np.uint32).reshape(cols, ldw)
    allr = np.arange(ldw * G)
    wi, k = allr // G, allr % G
    shift = (8 * (k % 4) + bits * (k // 4)).astype(np.uint32)
    codes = (w[:, wi] >> shift[None, :]) & np.uint32((1 << bits) - 1)
    return bool(np.all(codes[:, rows:] == 0))
