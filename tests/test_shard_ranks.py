"""The right-hand side split over the transfer momenta of one model (paper_1710_08830_gb300.shard) on CPU ranks:
gloo, world size 2.  Each rank holds the state rows of its own momenta, forms its part of the lattice Fourier
transform (Sec. 3.3), one all-reduce sums the parts, and each rank finishes its own rows (loops at its momenta,
projections from the summed transform, c A L A).  On the CPU the numbers come from the oracle, which implements the
same two steps (or_shard_transform, or_shard_finish), so these tests check the partition and the exchange and pin
the oracle's shard functions to its full right-hand side; the library's CUDA shard entry points are checked on the
GPU (tests/test_gpu_parity.py, shards emulated on one device)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MODELS = {
    "rashba_ff9": dict(kind="rashba", tp=-0.2, alpha=0.3, U=2.5, mu=-0.9, Lq=5, nc=2, n_ff=9),
    "t2g_ff5": dict(kind="t2g", seed=2, Lq=4, nc=1, n_ff=5, filling=4.0, T_mu=0.05),
}


def _spec(name):
    sys.path.insert(0, ROOT)
    from paper_1710_08830_gb300 import inputs
    kw = dict(MODELS[name])
    kind = kw.pop("kind")
    return inputs.rashba_hubbard(**kw) if kind == "rashba" else inputs.t2g_soc(**kw)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, name, mask, results):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["OMP_NUM_THREADS"] = "2"
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1710_08830_gb300 import inputs, shard
    oracle.set_threads(2)
    spec = _spec(name)
    o = oracle.Oracle(spec)
    state = inputs.random_state(spec, seed=5, scale=0.3)          # the same state on every rank
    q = shard.partition(spec.Nq, world, rank)
    local = np.ascontiguousarray(state[:, q])                     # this rank's rows only
    d_local = shard.sharded_rhs(o, 0.2, local, q, mask=mask)
    full = shard.gather_rows(d_local, q, spec.Nq).numpy()
    results[rank] = (q.tolist(), full)
    dist.destroy_process_group()


@pytest.mark.parametrize("name,mask", [("rashba_ff9", 3), ("rashba_ff9", 1), ("t2g_ff5", 3)])
def test_two_ranks_equal_the_whole_right_hand_side(name, mask):
    """Every rank's rows of the sharded right-hand side equal the oracle's unsharded right-hand side (1e-12
    relative); the two ranks' momenta partition the mesh."""
    import oracle
    from paper_1710_08830_gb300 import inputs
    world = 2
    with mp.Manager() as man:
        results = man.dict()
        mp.spawn(_worker, args=(world, _free_port(), name, mask, results), nprocs=world, join=True)
        res = dict(results)
    spec = _spec(name)
    qs = sorted(q for r in range(world) for q in res[r][0])
    assert qs == list(range(spec.Nq))
    assert 0 < len(res[0][0]) < spec.Nq
    ref, _ = oracle.Oracle(spec).rhs(0.2, inputs.random_state(spec, seed=5, scale=0.3), mask)
    for r in range(world):
        got = res[r][1]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


def test_partition_and_uneven_shards_in_one_process():
    """Without a process group the exchange is the identity: three uneven shards summed by hand give the whole
    right-hand side; the partition covers the mesh in contiguous blocks of sizes differing by at most one."""
    import oracle
    from paper_1710_08830_gb300 import inputs, shard
    spec = _spec("rashba_ff9")
    for world in (1, 2, 3, 7):
        parts = [shard.partition(spec.Nq, world, r) for r in range(world)]
        assert np.array_equal(np.concatenate(parts), np.arange(spec.Nq))
        assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        shard.partition(4, 5, 0)
    o = oracle.Oracle(spec)
    state = inputs.random_state(spec, seed=8, scale=0.3)
    shards = [np.array([0, 7, 3, 19]), np.arange(8, 15), np.array([q for q in range(spec.Nq) if q not in
                                                                  (0, 7, 3, 19) and not 8 <= q < 15])]
    xr = sum(o.shard_transform(state[:, s], s) for s in shards)
    ref, _ = o.rhs(0.35, state, 3)
    for s in shards:
        d = o.shard_finish(0.35, state[:, s], s, xr)
        assert np.abs(d - ref[:, s]).max() <= 1e-12 * np.abs(ref).max()
    # a shard alone does not see the other shards' part of the transform
    d0 = o.shard_finish(0.35, state[:, shards[1]], shards[1], o.shard_transform(state[:, shards[1]], shards[1]))
    assert np.abs(d0 - ref[:, shards[1]]).max() > 1e-3 * np.abs(ref).max()
