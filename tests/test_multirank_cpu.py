"""World-size-2 gloo ranks on the CPU: the source partition plus one sum
reproduces the single-rank misfit and gradient, and a rank that never reports
is dropped from the sum after the deadline (Sec. 3 worker-timeout proposal).
The per-rank work is the CPU oracle on a small 2D problem; no GPU is used."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import helmholtz as O
from paper_1703_09268_gb300 import parallel


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    rng = np.random.default_rng(4)
    n = 25
    g = O.make_grid(2, (n, 1, n), 25.0, (6, 0, 6), 2500.0)
    v = 2000 + 300 * rng.random((n, 1, n))
    mt = 1 / v ** 2
    m0 = np.full(g.phys_shape, 1 / 2150 ** 2)
    src = np.array([2 + n * 2, 8 + n * 2, 12 + n * 2, 18 + n * 2, 22 + n * 2], dtype=np.int32)
    Q = np.eye(5, dtype=complex)
    rec = (np.arange(n) + n * 1).astype(np.int32)
    freqs = np.array([4.0, 7.0])
    _, d = O.forward(g, mt, freqs, src, Q, rec)
    return g, m0, freqs, src, Q, rec, d


def _rank_work(rank, world, mask_pairs):
    g, m0, freqs, src, Q, rec, d = _problem()
    nf, ns = len(freqs), Q.shape[1]
    mine = parallel.shard(nf * ns, rank, world)
    mask = np.zeros((nf, ns), dtype=bool)
    for p in mine:
        if mask_pairs is None or p in mask_pairs:
            mask[p // ns, p % ns] = True
    f, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d, mask=mask)
    return f, gr


def _worker_allreduce(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    f, gr = _rank_work(rank, world, None)
    tf = torch.tensor([f], dtype=torch.float64)
    tg = torch.from_numpy(gr.ravel().copy())
    parallel.allreduce_sum([tf, tg])
    if rank == 0:
        np.save(out, np.concatenate([tf.numpy(), tg.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def _worker_deadline(rank, world, port, out):
    store = dist.TCPStore("127.0.0.1", port, world, rank == 0, timeout=__import__("datetime").timedelta(seconds=30))
    f, gr = _rank_work(rank, world, None)
    if rank == 1:
        return  # this worker "fails": it never publishes its contribution
    sums, got = parallel.sum_with_deadline(store, "step0", rank, world, [np.array([f]), gr.ravel()], 2.0)
    np.save(out, np.concatenate([sums[0], sums[1], np.array(got, dtype=float)]))


def test_shard_covers_every_pair_once():
    for units in (1, 5, 16, 17):
        for world in (1, 2, 3, 8):
            seen = sorted(sum((parallel.shard(units, r, world) for r in range(world)), []))
            assert seen == list(range(units))


def test_two_rank_allreduce_equals_single_rank(tmp_path):
    out = str(tmp_path / "ar.npy")
    mp.spawn(_worker_allreduce, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    g, m0, freqs, src, Q, rec, d = _problem()
    f, gr = O.misfit_and_gradient(g, m0, freqs, src, Q, rec, d)
    assert got[0] == pytest.approx(f, rel=1e-13)
    assert np.allclose(got[1:], gr.ravel(), rtol=1e-12, atol=1e-12 * np.abs(gr).max())


def test_late_rank_is_dropped_after_deadline(tmp_path):
    out = str(tmp_path / "dl.npy")
    mp.spawn(_worker_deadline, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    f0, g0 = _rank_work(0, 2, None)
    n = g0.size
    assert got[0] == pytest.approx(f0, rel=1e-13)
    assert np.allclose(got[1:1 + n], g0.ravel())
    assert list(got[1 + n:]) == [0.0]


def _worker_gn(rank, world, port, out):
    """Each rank applies the Gauss-Newton and full Hessian products on its
    share of the (frequency, source) pairs; one all-reduce sums them."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g, m0, freqs, src, Q, rec, d = _problem()
    nf, ns = len(freqs), Q.shape[1]
    mask = np.zeros((nf, ns), dtype=bool)
    for p in parallel.shard(nf * ns, rank, world):
        mask[p // ns, p % ns] = True
    dm = np.random.default_rng(5).standard_normal(g.n_phys) * 1e-8
    gn = O.gauss_newton_hessvec(g, m0, freqs, src, Q, rec, dm, mask=mask).ravel()
    hv = O.hessvec(g, m0, freqs, src, Q, rec, d, dm, mask=mask).ravel()
    t = [torch.from_numpy(gn.copy()), torch.from_numpy(hv.copy())]
    parallel.allreduce_sum(t)
    if rank == 0:
        np.save(out, np.concatenate([t[0].numpy(), t[1].numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_hessian_products_equal_single_rank(tmp_path):
    """The linearised calls shard like the gradient: per-pair sums plus one
    all-reduce (Gauss-Newton and full Hessian products)."""
    out = str(tmp_path / "gn.npy")
    mp.spawn(_worker_gn, args=(2, _free_port(), out), nprocs=2, join=True)
    got = np.load(out)
    g, m0, freqs, src, Q, rec, d = _problem()
    dm = np.random.default_rng(5).standard_normal(g.n_phys) * 1e-8
    gn = O.gauss_newton_hessvec(g, m0, freqs, src, Q, rec, dm).ravel()
    hv = O.hessvec(g, m0, freqs, src, Q, rec, d, dm).ravel()
    n = gn.size
    assert np.allclose(got[:n], gn, rtol=1e-12, atol=1e-12 * np.abs(gn).max())
    assert np.allclose(got[n:], hv, rtol=1e-12, atol=1e-12 * np.abs(hv).max())


def test_bench_step_sources_partition_the_multifrequency_workload():
    """bench.py's rank-r step takes its own sources of the 192^3 recipe (same
    8 x 16 source grid at any size): distinct across ranks, the centre source
    first on rank 0, and each source's point (node index, unit weight) kept."""
    import bench
    from paper_1703_09268_gb300 import synth
    wl = synth.workload_3d_multifreq(n=32)
    s0 = synth.centre_source(wl)
    nx, ny, _ = wl.n
    loc = wl.src_idx[s0]
    assert abs(loc % nx - (nx - 1) / 2) <= nx / 8 and abs((loc // nx) % ny - (ny - 1) / 2) <= ny / 8
    for world in (1, 2, 4, 8):
        for k in (1, 2):
            cols = [c for r in range(world) for c in bench.step_columns(wl, r, k)]
            assert len(set(cols)) == world * k and cols[0] == s0
    src, Q = synth.source_subset(wl, [s0, (s0 + 1) % wl.nsrc])
    assert list(src) == [wl.src_idx[s0], wl.src_idx[(s0 + 1) % wl.nsrc]]
    assert np.array_equal(Q, np.eye(2))
