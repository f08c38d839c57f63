"""GPU parity of the block-sparse storage (NSRGS_BCSR_F32 / NSRGS_BCSR_BF16) for
incomplete observations (§4.1: pairs observed with probability p, unobserved
A_ij = 0): packed size, the product A_off X against float64, whole solves and
the objective against the oracle.
"""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import __graft_entry__

    __graft_entry__.build()
    import paper_2604_07372_gb300 as P

    return P


def to64(t):
    return t.detach().double().cpu().numpy()


def observed_blocks(inst):
    return int(np.count_nonzero(np.any(inst.upper.reshape(len(inst.upper), -1) != 0, axis=1)))


CASES = [(2, 3, 1.0), (3, 1, 0.5), (70, 3, 0.3), (257, 4, 0.05), (50, 3, 0.01), (1000, 3, 0.2), (120, 8, 0.4),
         (200, 2, 1.0)]


@pytest.mark.parametrize("storage", ["bcsr_f32", "bcsr_bf16"])
@pytest.mark.parametrize("n,d,p", CASES)
def test_bcsr_product_matches_dense_matmul(P, n, d, p, storage):
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=n + d, p=p, dtype=np.float32)
    A = inst.dense()
    for i in range(n):
        A[i * d : (i + 1) * d, i * d : (i + 1) * d] = 0.0
    up = torch.from_numpy(inst.upper).cuda()
    st = P.STORAGE[storage]
    nnzb = 2 * observed_blocks(inst)
    E = 4 if storage == "bcsr_f32" else 2
    nb = P.nsrgs_bcsr_packed_bytes(up, n, d, st)
    # values in groups of 32 blocks, the last group zero-padded
    assert nb >= nnzb * d * d * E and nb <= nnzb * (d * d * E + 4) + 31 * d * d * E + 8 * (n + 1) + 64 + 3 * 256
    pa = P.nsrgs_pack_upper(up, n, d, st)
    X = np.random.default_rng(n).standard_normal((n * d, d)).astype(np.float32)
    Y = P.nsrgs_product(pa, torch.from_numpy(X).cuda())
    torch.cuda.synchronize()
    if storage == "bcsr_bf16":
        A = torch.from_numpy(A).to(torch.bfloat16).to(torch.float64).numpy()
    ref = A @ X.astype(np.float64)
    scale = np.abs(A) @ np.abs(X.astype(np.float64))
    assert np.all(np.abs(to64(Y) - ref) <= 1e-6 * scale + 1e-6)


@pytest.mark.parametrize("n,d,p,storage", [(70, 3, 0.3, "bcsr_f32"), (45, 2, 0.6, "bcsr_bf16"), (33, 5, 0.5, "bcsr_f32")])
def test_bcsr_buffer_follows_the_documented_layout(P, n, d, p, storage):
    """Header, int64 row pointers, int32 columns in increasing j, values in groups of
    32 blocks interleaved element by element (element e of block k at
    32*d*d*(k//32) + 32*e + k%32), zero padding after the last stored block."""
    inst = synth.make_instance(n, d, 1.0, seed=n * d, p=p, dtype=np.float32)
    A = inst.dense()
    st = P.STORAGE[storage]
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, st)
    torch.cuda.synchronize()
    buf = pa.buf.cpu().numpy()
    hdr = buf[:64].view(np.int64)
    nnzb, off_col, off_val = int(hdr[2]), int(hdr[3]), int(hdr[4])
    assert (hdr[0], hdr[1]) == (n, d) and off_col % 16 == 0 and off_val % 16 == 0
    rowptr = buf[64 : 64 + 8 * (n + 1)].view(np.int64)
    col = buf[off_col : off_col + 4 * nnzb].view(np.int32)
    dt = np.float32 if storage == "bcsr_f32" else np.uint16
    E = 4 if storage == "bcsr_f32" else 2
    slots = (nnzb + 31) // 32 * 32
    raw = buf[off_val : off_val + slots * d * d * E].view(dt)
    vals = raw.astype(np.float32) if E == 4 else (raw.astype(np.uint32) << 16).view(np.float32)
    expect_cols = []
    for i in range(n):
        for j in range(n):
            blk = A[i * d : (i + 1) * d, j * d : (j + 1) * d]
            if j != i and np.any(blk != 0):
                expect_cols.append((i, j))
    assert nnzb == len(expect_cols) and rowptr[0] == 0 and rowptr[n] == nnzb
    for k, (i, j) in enumerate(expect_cols):
        assert rowptr[i] <= k < rowptr[i + 1] and col[k] == j
        pos = 32 * d * d * (k // 32) + 32 * np.arange(d * d) + k % 32
        ref = A[i * d : (i + 1) * d, j * d : (j + 1) * d].reshape(-1)
        if E == 2:
            ref = torch.from_numpy(ref.copy()).to(torch.bfloat16).float().numpy()
        assert np.array_equal(vals[pos], ref)
    used = np.zeros(slots * d * d, dtype=bool)
    for k in range(nnzb):
        used[32 * d * d * (k // 32) + 32 * np.arange(d * d) + k % 32] = True
    assert np.all(vals[~used] == 0.0)
    assert np.all(buf[off_val + slots * d * d * E :] == 0)


def test_bcsr_from_dense_equals_from_upper(P):
    n, d, p = 150, 3, 0.25
    inst = synth.make_instance(n, d, 1.0, seed=4, p=p, dtype=np.float32)
    Ad = torch.from_numpy(inst.dense(dtype=np.float32)).cuda()
    up = torch.from_numpy(inst.upper).cuda()
    a = P.nsrgs_pack_upper(up, n, d, P.BCSR_F32)
    b = P.nsrgs_pack_dense(Ad, n, d, P.BCSR_F32)
    torch.cuda.synchronize()
    assert a.nbytes == b.nbytes and torch.equal(a.buf, b.buf)


@pytest.mark.parametrize("n,d,p", [(300, 3, 0.2), (200, 4, 0.5)])
def test_bcsr_solve_matches_oracle(P, n, d, p):
    T, K = 30, 2
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=11 + d, p=p, dtype=np.float32)
    A = inst.dense()
    X0, _ = O.spectral_init(A, n, d)
    Xo, _ = O.nsrgs(A, n, d, 1.0 / n, T, K, X0=X0)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BCSR_F32)
    X, info = P.nsrgs_solve(pa, 1.0 / n, T, K, spectral_max_iters=100)
    torch.cuda.synchronize()
    assert info.iters == T
    assert O.dF(to64(X), Xo, d) / math.sqrt(n * d) <= 1e-5


def test_bcsr_objective_matches_oracle(P):
    n, d, p = 250, 3, 0.3
    inst = synth.make_instance(n, d, synth.sigma_rule(0.3, n, d), seed=21, p=p, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BCSR_F32)
    X = inst.Zstack().astype(np.float32)
    F = P.nsrgs_objective(pa, torch.from_numpy(X).cuda())
    ref = O.objective(inst.dense(), X.astype(np.float64), n, d)
    assert abs(F - ref) <= 1e-5 * abs(ref)


def test_bcsr_is_refused_where_not_built(P):
    inst = synth.make_instance(20, 9, 0.5, seed=1, p=0.5, dtype=np.float32)
    with pytest.raises(P.NsrgsError):
        P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), 20, 9, P.BCSR_F32)


@pytest.mark.parametrize("d,storage", [(3, "bcsr_f32"), (4, "bcsr_bf16")])
def test_corrupted_row_pointer_is_reported_not_faulted(P, d, storage):
    """A row pointer past the stored blocks is caught by the row kernel's own
    check (the row is skipped) and the solve returns INVALID_ARG."""
    n = 60
    inst = synth.make_instance(n, d, 1.0, seed=5, p=0.5, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.STORAGE[storage])
    torch.cuda.synchronize()
    nnzb = int(pa.buf[:64].cpu().numpy().view(np.int64)[2])
    bad = np.array([nnzb + 1000], dtype=np.int64).view(np.uint8)
    pa.buf[64 + 8 * 5 : 64 + 8 * 6] = torch.from_numpy(bad.copy()).cuda()  # rowptr[5]
    with pytest.raises(P.NsrgsError) as e:
        P.nsrgs_solve(pa, 1.0 / n, 3, 2, spectral_max_iters=5)
        torch.cuda.synchronize()
    assert e.value.status == 1  # NSRGS_ERR_INVALID_ARG


def test_corrupted_column_index_stays_in_bounds(P):
    """A stored column index outside [0, n) is clamped into range by the row
    kernel: the solve runs to completion (wrong data in, but no fault)."""
    n, d = 60, 3
    inst = synth.make_instance(n, d, 1.0, seed=5, p=0.5, dtype=np.float32)
    pa = P.nsrgs_pack_upper(torch.from_numpy(inst.upper).cuda(), n, d, P.BCSR_F32)
    torch.cuda.synchronize()
    off_col = int(pa.buf[:64].cpu().numpy().view(np.int64)[3])
    bad = np.array([n + 100000], dtype=np.int32).view(np.uint8)
    pa.buf[off_col : off_col + 4] = torch.from_numpy(bad.copy()).cuda()
    X, info = P.nsrgs_solve(pa, 1.0 / n, 3, 2, spectral_max_iters=5)
    torch.cuda.synchronize()
    assert info.iters == 3 and torch.isfinite(X).all()
