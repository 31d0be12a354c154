"""Slab decomposition on CPU (no GPU): the partition and the transposes of
paper_2306_04322_gb300.slab against the oracle, over gloo with world sizes 2
and 4 (127.0.0.1).

Each rank runs the two halves of Algorithm 1's step on its share in FP64
numpy -- test-side executors that keep the library's packed layout (row
spectra [slot][y][kx], column 0 holding the real kx = 0 and kx = nx/2
spectra as real and imaginary parts; the column pass separates them on the
rank that owns column 0) -- and moves every block with the module's
exchange_forward / exchange_back.  The pointwise derivatives and |xi|^2
come from the oracle; the y transforms see only this rank's columns.  After
k steps the gathered fields must equal the oracle's Algorithm 1 to rounding:
a block sent to the wrong rank, row range or slot, or a column given the
wrong global kx, fails it.
"""
import dataclasses
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2306_04322_gb300 import inputs as I  # noqa: E402
from paper_2306_04322_gb300 import slab as S  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def pack(X):
    """rfft output (..., nx/2 + 1) -> packed half spectrum (..., nx/2)."""
    P = X[..., :-1].copy()
    P[..., 0] = X[..., 0].real + 1j * X[..., -1].real
    return P


def unpack(P):
    H = P.shape[-1]
    X = np.zeros(P.shape[:-1] + (H + 1,), dtype=complex)
    X[..., 1:H] = P[..., 1:]
    X[..., 0] = P[..., 0].real
    X[..., H] = P[..., 0].imag
    return X


def as_real(z):
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.stack([z.real, z.imag], axis=-1)))


def as_cplx(t):
    a = t.numpy()
    return a[..., 0] + 1j * a[..., 1]


def row_pass(O, pr, lay, u):
    """Real rows u (nf, rows, nx) -> packed x spectra of c, g_i, df/dc."""
    sub = dataclasses.replace(pr, n=(pr.n[0], lay.rows))
    d = O.derivatives(sub, u)
    slots = [u[0]] + [u[i] - pr.L * pr.dt * d[i] for i in range(1, pr.nf)] + [d[0]]
    return pack(np.fft.rfft(np.stack(slots), axis=-1))


def col_pass(O, pr, lay, colspec):
    """Column spectra (slots_fwd, ny, cols) -> new c, eta_i (nf, ny, cols)."""
    nx, ny = pr.n
    K2 = O.k2(pr)  # (ny, nx)
    Z = np.fft.fft(colspec, axis=1)
    k0 = lay.col_range().start
    k2 = K2[:, k0:k0 + lay.cols]

    def solve(f, zf, zc, kk):
        if f == 0:
            return (zc - pr.M * pr.dt * kk * zf) / (1.0 + pr.M * pr.dt * pr.kappa_c * kk * kk)
        return zc / (1.0 + pr.L * pr.dt * pr.kappa_eta * kk)

    out = np.empty((pr.nf, ny, lay.cols), dtype=complex)
    zf = Z[pr.nf]
    for f in range(pr.nf):
        out[f] = solve(f, zf, Z[f], k2)
        if k0 == 0:
            # packed column: A (kx = 0) and B (kx = nx/2), both Hermitian in ky
            def split(z):
                zr = np.conj(np.roll(z[::-1], 1))
                return 0.5 * (z + zr), -0.5j * (z - zr)
            A, B = split(Z[f][:, 0])
            Af, Bf = split(zf[:, 0])
            out[f][:, 0] = solve(f, Af, A, K2[:, 0]) + 1j * solve(f, Bf, B, K2[:, nx // 2])
    return np.fft.ifft(out, axis=1)


def _rank_main(rank, world, port, n, p, nsteps, out_dir):
    import torch
    import torch.distributed as dist
    from oracle import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    pr = I.Problem(n=n, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    lay = S.SlabLayout(n[0], n[1], p, world, rank)
    u = I.noise_fields(pr, seed=31)[:, lay.row_range()].copy()
    send = torch.zeros((world, lay.slots_fwd, lay.rows, lay.cols, 2), dtype=torch.float64)
    recv = torch.zeros((world, lay.slots_back, lay.rows, lay.cols, 2), dtype=torch.float64)
    colspec = torch.zeros((lay.slots_fwd, n[1], lay.cols, 2), dtype=torch.float64)
    for _ in range(nsteps):
        spec = row_pass(O, pr, lay, u)
        for q in range(world):
            blk = as_real(spec[:, :, lay.col_range(q)])
            if q == rank:
                colspec[:, lay.row_range()] = blk
            else:
                send[q] = blk
        S.exchange_forward(lay, send, colspec, dist)
        new = col_pass(O, pr, lay, as_cplx(colspec))
        colspec[:lay.slots_back] = as_real(new)
        S.exchange_back(lay, colspec, recv, dist)
        P = np.empty((pr.nf, lay.rows, n[0] // 2), dtype=complex)
        for q in range(world):
            P[:, :, lay.col_range(q)] = as_cplx(colspec[:lay.slots_back, lay.row_range()] if q == rank else recv[q])
        u = np.fft.irfft(unpack(P), n=n[0], axis=-1)
    np.save(os.path.join(out_dir, f"rank{rank}.npy"), u)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,n,p", [(2, (32, 16), 2), (4, (32, 32), 1), (2, (16, 64), 0)])
def test_slab_transposes_match_the_oracle(O, tmp_path, world, n, p):
    mp = pytest.importorskip("torch.multiprocessing")
    nsteps = 3
    mp.start_processes(_rank_main, args=(world, _free_port(), n, p, nsteps, str(tmp_path)), nprocs=world,
                       start_method="spawn")
    got = np.concatenate([np.load(tmp_path / f"rank{r}.npy") for r in range(world)], axis=1)
    pr = I.Problem(n=n, p=p)
    pr.dt = 5.0 * I.fd_stable_dt(pr)
    ref, _ = O.step(pr, I.noise_fields(pr, seed=31), nsteps)
    err = max(np.max(np.abs(got[f] - ref[f])) / np.max(np.abs(ref[f])) for f in range(pr.nf))
    assert err <= 1e-12, err


def test_layout_partitions_the_grid():
    for R in (1, 2, 4, 8):
        lays = [S.SlabLayout(128, 64, 2, R, r) for r in range(R)]
        rows = np.concatenate([np.arange(64)[l.row_range()] for l in lays])
        cols = np.concatenate([np.arange(64)[l.col_range()] for l in lays])
        assert (rows == np.arange(64)).all() and (cols == np.arange(64)).all()
        fwd, back = lays[0].exchange_bytes(8)
        assert fwd == (R - 1) * 4 * (64 // R) * (64 // R) * 8
        assert back == (R - 1) * 3 * (64 // R) * (64 // R) * 8
    for bad in [dict(nranks=3, rank=0), dict(nranks=2, rank=2), dict(nranks=16, rank=0)]:
        with pytest.raises(ValueError):
            S.SlabLayout(128, 64, 2, **bad)
