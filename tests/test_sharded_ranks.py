"""The paper's row-block distributed CGD-EnKF (Sec. 3.3) on CPU ranks (gloo, world sizes 2
and 3): observation rows of HA, D and the CG vectors split in contiguous blocks, the
matvec's stage 1 summed by an allreduce, the CG column sums by allreduces, W replicated and
each rank updating its own block of state rows. The assembled X_a equals the single-process
CG of the oracle at fixed step counts (round-off only: sums run in another order) and the
exact analysis when converged, for diagonal and tridiagonal R (whose stage 3 needs each
neighbour's boundary rows)."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import sharded
import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(tri):
    rng = np.random.default_rng(5)
    n, N, m = 90, 12, 37
    Xf = rng.standard_normal((n, N)) + 2.0 * rng.standard_normal(n)[:, None]
    rowptr, col, w = [0], [], []
    for _ in range(m):
        k = int(rng.integers(1, 4))
        col += list(rng.choice(n, size=k, replace=False))
        w += list(rng.uniform(-1.5, 1.5, size=k))
        rowptr.append(len(col))
    r = rng.uniform(0.3, 2.0, size=m)
    r_off = 0.3 * np.minimum(r[:-1], r[1:]) if tri else None
    y = rng.standard_normal(m)
    E = rng.standard_normal((m, N))
    return Xf, np.array(rowptr, np.int32), np.array(col, np.int32), np.array(w), r, r_off, y, E


def _worker(rank, ws, port, out_dir, tri, fixed):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        def allreduce(a):
            t = torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64))
            dist.all_reduce(t)
            return t.numpy()

        Xf, rowptr, col, w, r, r_off, y, E = _problem(tri)
        Xa, (lo, hi), info = sharded.cgd_enkf_rowblock(Xf, rowptr, col, w, r, y, rank, ws, allreduce, E=E,
                                                       tol=1e-12, fixed_iters=fixed, r_off=r_off)
        np.save(os.path.join(out_dir, f"x{rank}.npy"), Xa)
        np.save(os.path.join(out_dir, f"rows{rank}.npy"), np.array([lo, hi]))
        np.save(os.path.join(out_dir, f"it{rank}.npy"), info["iters"])
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run(tmp_path, ws, tri, fixed):
    mp.start_processes(_worker, args=(ws, _free_port(), str(tmp_path), tri, fixed), nprocs=ws, join=True,
                       start_method="spawn")
    parts, its = [], []
    for k in range(ws):
        lo, hi = np.load(tmp_path / f"rows{k}.npy")
        parts.append((lo, hi, np.load(tmp_path / f"x{k}.npy")))
        its.append(np.load(tmp_path / f"it{k}.npy"))
    n = max(hi for _, hi, _ in parts)
    Xa = np.zeros((n, parts[0][2].shape[1]))
    for lo, hi, x in parts:
        Xa[lo:hi] = x
    assert all(np.array_equal(its[0], i) for i in its)     # every rank takes the same decisions
    return Xa, its[0]


@pytest.mark.parametrize("ws", [2, 3])
@pytest.mark.parametrize("tri", [False, True])
def test_row_block_cg_equals_single_process_cg(tmp_path, ws, tri):
    Xf, rowptr, col, w, r, r_off, y, E = _problem(tri)
    # fixed step counts: the iterates must agree to round-off
    Xa, _ = _run(tmp_path, ws, tri, fixed=4)
    ref, _ = oracle.cgd_enkf(Xf, rowptr, col, w, r, y, E, fixed_iters=4, r_off=r_off)
    assert oracle.rel_frobenius(Xa, ref) <= 1e-12
    # converged: the exact analysis (dense Cholesky of the full S, Algorithm 1)
    Xa, it = _run(tmp_path, ws, tri, fixed=0)
    exact = oracle.enkf_alg1(Xf, rowptr, col, w, r, y, E, r_off=r_off)
    assert oracle.rel_frobenius(Xa, exact) <= 1e-9
    assert it.max() > 4


def test_row_blocks_cover_the_rows_once():
    for count in (1, 7, 37, 64):
        for size in (1, 2, 3, 5):
            blocks = [sharded.row_block(count, k, size) for k in range(size)]
            assert blocks[0][0] == 0 and blocks[-1][1] == count
            assert all(b[1] == c[0] for b, c in zip(blocks[:-1], blocks[1:]))
