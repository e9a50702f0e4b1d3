"""Lag sharding (Section 3 distribution, one lag block per unit) on the CPU:
the partition of stbem_lag_shard (host code of the library, no GPU), and two
gloo ranks whose partial products, computed by the oracle over each rank's
lags only, are summed by the library's all-reduce callback adaptor
(shard.make_allreduce_callback over torch.distributed) into the full product,
and drive a GMRES to the oracle's block forward substitution."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")
mp = pytest.importorskip("torch.multiprocessing")


def _work(nt, n_ranks, rank, chunk):
    from paper_1811_05224_gb300 import shard
    return sum((nt - d) for a, b in shard.lag_ranges(nt, n_ranks, rank, chunk) for d in range(a, b))


@pytest.mark.parametrize("nt,n_ranks,chunk", [(1, 1, 16), (5, 3, 1), (100, 4, 16), (256, 8, 16), (1024, 8, 16),
                                              (1024, 3, 32), (40, 8, 16), (513, 2, 7)])
def test_lag_partition_covers_every_lag_once_and_balances(nt, n_ranks, chunk):
    from paper_1811_05224_gb300 import shard
    seen = np.zeros(nt, dtype=int)
    for r in range(n_ranks):
        ranges = shard.lag_ranges(nt, n_ranks, r, chunk)
        prev = -1
        for a, b in ranges:
            assert 0 <= a < b <= nt and a > prev       # increasing, disjoint, merged (a > previous end)
            seen[a:b] += 1
            prev = b
    assert np.all(seen == 1)
    # work sum (nt - d) per rank: within one chunk's largest work of the mean
    # when every rank receives at least two rounds of chunks
    nchunks = -(-nt // chunk)
    if nchunks >= 2 * n_ranks:
        works = [_work(nt, n_ranks, r, chunk) for r in range(n_ranks)]
        mean = nt * (nt + 1) / 2 / n_ranks
        assert max(abs(w - mean) for w in works) <= chunk * nt


def test_lag_partition_rejects_bad_arguments():
    import ctypes
    from paper_1811_05224_gb300 import capi
    lib = capi.load()
    buf = (ctypes.c_int * 4)()
    n = ctypes.c_int()
    assert lib.stbem_lag_shard(0, 2, 0, 16, 2, buf, ctypes.byref(n)) == capi.STBEM_ERR_ARG
    assert lib.stbem_lag_shard(10, 2, 2, 16, 2, buf, ctypes.byref(n)) == capi.STBEM_ERR_ARG
    # chunks 0, 3-4, 7-8, 11-12, 15: 5 ranges, room for 2: NOMEM and the count
    assert lib.stbem_lag_shard(64, 2, 0, 4, 2, buf, ctypes.byref(n)) == capi.STBEM_ERR_NOMEM
    assert n.value == 5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    import workloads as W
    from oracle import assembly as OA
    from oracle.geometry import BoundaryMesh
    om = BoundaryMesh(W.l_shape(16, seed=3), 1.0, 12, 0.5)
    return om, OA.assemble("V", om), OA.assemble("D", om), OA.lumped_dual_mass(om)


def _rank(rank, world, port, out):
    from oracle import solve as OS
    from paper_1811_05224_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        om, V, D, Lm = _problem()
        nt = V.shape[0]
        ranges = shard.lag_ranges(nt, world, rank, 4)
        mask = np.zeros(nt, dtype=bool)
        for a, b in ranges:
            mask[a:b] = True
        Vr, Dr = V * mask[:, None, None], D * mask[:, None, None]     # this rank's blocks only
        # the reduction goes through the library's callback adaptor on a
        # workspace-like buffer, at an offset, as the solver calls it
        buf = torch.zeros(64 + 8 * V.shape[0] * V.shape[1] + 64, dtype=torch.uint8)
        cb = shard.make_allreduce_callback(buf, shard.default_reducer())
        region = buf[64:64 + 8 * nt * V.shape[1]].view(torch.float64)

        def reduced(partial):
            region.copy_(torch.from_numpy(partial.ravel()))
            assert cb(buf.data_ptr() + 64, region.numel(), None) == 0
            return region.numpy().reshape(partial.shape).copy()

        rng = np.random.default_rng(8)
        x = rng.standard_normal((nt, V.shape[1]))
        full = OS.toeplitz_apply(V, x)
        y = reduced(OS.toeplitz_apply(Vr, x))
        yt = reduced(OS.toeplitz_apply(Vr, x, transpose=True))
        err = max(np.abs(y - full).max() / np.abs(full).max(),
                  np.abs(yt - OS.toeplitz_apply(V, x, transpose=True)).max() / np.abs(full).max())
        # GMRES with the sharded products (V, and D in the preconditioner)
        f = OS.toeplitz_apply(V, rng.standard_normal((nt, V.shape[1])))

        def A(v):
            return reduced(OS.toeplitz_apply(Vr, v))

        def M(v):
            return reduced(OS.toeplitz_apply(Dr, v / Lm)) / Lm
        w, it, _ = OS.gmres(A, f, M, tol=1e-11)
        w_ref = OS.forward_substitution(V, f)
        out[rank] = (err, float(np.linalg.norm(w - w_ref) / np.linalg.norm(w_ref)), it, ranges)
        # a callback pointer outside its buffer is refused (STBEM_ERR_REDUCE upstream)
        assert cb(buf.data_ptr() + buf.numel(), 4, None) != 0
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_products_and_gmres():
    world, port = 2, _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
    covered = sorted(r for k in range(world) for r in out[k][3])
    assert covered[0][0] == 0 and covered[-1][1] == 12
    for r in range(world):
        err, werr, it, ranges = out[r]
        assert ranges, r                     # both ranks hold lags
        assert err <= 1e-14, (r, err)
        assert werr <= 1e-9, (r, werr)
    assert out[0][2] == out[1][2]            # the same iterations on both ranks
