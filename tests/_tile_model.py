"""NumPy model of the tile-upper layout of the tensor-core symmetric stream
(d in {16, 32, 64}): 128 x 128 tiles (I, J), J >= I, stored in the kernel's
processing order, each tile in the 128-byte-swizzled order the tensor core
reads.  Shared by the host layout checks and the GPU byte-level tests."""
import numpy as np

T = 128


def width(d):
    """Tile width (the MMA's N) for block size d: d rounded up to 16, 32 or 64."""
    return 16 if d <= 16 else (32 if d <= 32 else 64)


def strip_rows(d, f8=False):
    """Row tiles per strip / group of the processing order (FP8 at d = 32 keeps
    its hi and lo accumulators side by side, so fewer fit in TMEM); by tile width."""
    w = width(d)
    return 4 if w == 64 else (6 if f8 and w == 32 else 8)


def swz(r, c):
    """Byte offset of bfloat16 element (r, c) in a swizzled 128 x 128 tile."""
    s, k, e = c >> 6, (c & 63) >> 3, c & 7
    return (r >> 3) * 2048 + s * 1024 + (r & 7) * 128 + ((k ^ (r & 7)) << 4) + e * 2


def swz8(r, c):
    """Byte offset of one-byte element (r, c) in a swizzled 128-column tile (any row count)."""
    return (r >> 3) * 1024 + (r & 7) * 128 + (((c >> 4) ^ (r & 7)) << 4) + (c & 15)


def sw128(addr):
    """The 128-byte swizzle as an address map: bits [4:6] ^= bits [7:9]."""
    return addr ^ (((addr >> 7) & 7) << 4)


def order(NT, R):
    """The processing (and storage) order: (I, J) of every stored tile."""
    out = []
    for g in range(-(-NT // R)):
        I0 = g * R
        Rg = min(R, NT - I0)
        for J in range(I0, NT):
            for r in range(min(Rg, J - I0 + 1)):
                out.append((I0 + r, J))
    return out


def seek(t, NT, R):
    """Position t -> (I, J) as the kernel and the packer compute it."""
    base, g = 0, 0
    while True:
        L = NT - g * R
        Rg = min(R, L)
        cnt = Rg * (Rg + 1) // 2 + (L - Rg) * Rg
        if t < base + cnt:
            break
        base += cnt
        g += 1
    I0, Rg = g * R, min(R, NT - g * R)
    u = t - base
    tri = Rg * (Rg + 1) // 2
    if u < tri:
        c = 0
        while u >= c + 1:
            u -= c + 1
            c += 1
        return I0 + u, I0 + c
    u -= tri
    return I0 + u % Rg, I0 + Rg + u // Rg


def tile_rows(n, d):
    return -(-(n * d) // T)


def fp8_tile_bytes(n, d):
    """Packed bytes of the FP8 tile-upper layout: 16 KB tiles, then n float32 scales (16-byte padded)."""
    NT = tile_rows(n, d)
    return NT * (NT + 1) // 2 * 16384 + (4 * n + 15) // 16 * 16


def pow2_scale(m):
    """Operand scale of the FP8 product: g = 2^(7 - floor(log2 m)), so m g lies in [128, 256);
    g = 1 for m = 0; the exponent clamped to [-100, 120]."""
    m = np.float32(m)
    if m == 0:
        return np.float32(1.0)
    e = int(np.frexp(m)[1]) - 1
    e = max(-100, min(e, 120))
    return np.float32(2.0 ** (7 - e))
