"""NumPy model of the symmetric panel layout (slabs, steps, stored warp slices,
the [w][rt][lane][cc] order inside a slice), shared by the CPU layout tests and
the GPU test that reads packed bytes back.  It restates the layout from its
definition (rows per thread, bytes per load and consumer warps per (d, storage))
independently of the library's own tables."""
import numpy as np

E_OF = {0: 4, 1: 2, 2: 1}
# scalar rows per thread, per d
RT_OF = {1: 8, 2: 8, 3: 6, 4: 8, 5: 5, 6: 6, 7: 7, 8: 6}


def loadb(d, storage):
    """Bytes one thread loads per row and step."""
    if storage == 2:
        return 8
    if d <= 4:
        return 16
    if d == 7:
        return 8 if storage == 0 else 4
    return 16 if storage == 0 else 8


def nw(d, storage):
    """Consumer warps per CTA: 12 at d <= 2 and for FP32 at d = 3, else 8."""
    return 12 if (d <= 2 or (d == 3 and storage == 0)) else 8


class Geom:
    def __init__(self, n, d, storage):
        self.n, self.D, self.st = n, d, storage
        self.E = E_OF[storage]
        self.RT = 12 if (d == 3 and storage != 0) else RT_OF[d]
        self.LOADB = loadb(d, storage)
        self.CPT = self.LOADB // self.E
        self.SC = 4 * self.CPT
        self.NW = nw(d, storage)
        self.WROWS = 8 * self.RT
        self.RS = self.NW * self.WROWS
        assert self.RS % d == 0
        self.SB = self.RS // d
        self.WB = self.WROWS * self.SC * self.E
        self.nslabs = -(-n // self.SB)

    def warps(self, b, q):
        c_end = b * self.SB * self.D + (q + 1) * self.SC
        jmax = min((c_end - 1) // self.D, self.n - 1)
        rmax = (jmax - b * self.SB) * self.D
        rmax = min(rmax, (self.n - b * self.SB) * self.D, self.RS)
        rmax = max(rmax, 1)
        return min(-(-rmax // self.WROWS), self.NW)

    def steps(self, b):
        L = self.n * self.D - b * self.SB * self.D
        return -(-L // self.SC)

    def header_bytes(self):
        hdr = 16 * (self.nslabs + 1) + (4 * self.n if self.st == 2 else 0)
        return -(-hdr // 256) * 256

    def panel_bytes(self):
        return sum(self.warps(b, q) * self.WB for b in range(self.nslabs) for q in range(self.steps(b)))


def walk(g):
    """Yield (b, q, W, byte offset) in storage order."""
    off = 0
    for b in range(g.nslabs):
        for q in range(g.steps(b)):
            W = g.warps(b, q)
            yield b, q, W, off
            off += W * g.WB


def slot_coords(g, b, q, W):
    """Global (row, col) of every stored element of step (b, q), in storage order."""
    per = g.LOADB // g.E
    e = np.arange(W * g.WB // g.E)
    cc = e % per
    t = e // per
    lane = t % 32
    t //= 32
    rt = t % g.RT
    w = t // g.RT
    rg, cg = lane >> 2, lane & 3
    r = w * g.WROWS + rg * g.RT + rt
    c = cg * g.CPT + cc
    return b * g.SB * g.D + r, b * g.SB * g.D + q * g.SC + c
