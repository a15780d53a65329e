"""Several ranks (gloo, CPU): shift sharding plus one all-reduce of the reuse
sums reproduces the single-process sums exactly, and the estimator from the
joined sums (library host code) matches the oracle's."""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
import workloads as W

torch = pytest.importorskip("torch")
M = pytest.importorskip("paper_1806_05619_gb300")
from paper_1806_05619_gb300 import distributed as D  # noqa: E402

CFG = W.scaled(W.LATTICE_6LEVEL, n_levels=4, s=12, R=4, log2_nmax=6)
WORK = [(0, 0, 9, 0, 4), (1, 2, 6, 1, 4), (2, 0, 3, 0, 3), (3, 0, 2, 2, 4)]


def _oracle(mu0=None):
    z, _ = O.cbc(CFG["s"], CFG["log2_nmax"])
    return O.Oracle(n_levels=CFG["n_levels"], n0=CFG["n0"], s=CFG["s"], sigma=CFG["sigma"],
                    corr_len=CFG["corr_len"], qoi=CFG["qoi"], mu0=mu0 or CFG["mu0"], nu1=CFG["nu1"], nu2=CFG["nu2"],
                    sampler=CFG["sampler"], seed=CFG["seed"], R=CFG["R"], genvec=z, log2_nmax=CFG["log2_nmax"],
                    reuse=True)


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    orc = _oracle()
    mine = D.shard_work(WORK, CFG["R"], rank, world)
    sums = orc.sample_levels(mine)["sums"] if mine else np.zeros((CFG["n_levels"], CFG["R"], 2))
    t = torch.from_numpy(np.ascontiguousarray(sums).reshape(-1).copy())
    D.allreduce_sums(t)
    if rank == 0:
        np.save(out, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_shift_ranges_partition():
    for R in (1, 3, 16):
        for world in (1, 2, 3, 5):
            got = []
            for rank in range(world):
                r0, r1 = D.shift_range(R, rank, world)
                got += list(range(r0, r1))
            assert got == list(range(R))
    parts = [D.shard_work(WORK, CFG["R"], k, 3) for k in range(3)]
    n = sum((ne - nb) * (re_ - rb) for p in parts for (_, nb, ne, rb, re_) in p)
    assert n == sum((ne - nb) * (re_ - rb) for (_, nb, ne, rb, re_) in WORK)


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_sums_equal_single_process(world):
    import socket

    import torch.multiprocessing as mp

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = os.path.join(tempfile.mkdtemp(), "sums.npy")
    mp.start_processes(_rank, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    joined = np.load(out).reshape(CFG["n_levels"], CFG["R"], 2)
    orc = _oracle()
    want = orc.sample_levels(WORK)["sums"]
    assert np.array_equal(joined, want)
    N = [0] * CFG["n_levels"]
    for (lv, nb, ne, rb, re_) in WORK:
        N[lv] += (ne - nb) * (re_ - rb)
    # N of the estimator: samples per shift ending at each level (nominal here:
    # both sides get the same counts, the check is of the joined formula)
    Nr = [max(1, n // CFG["R"]) for n in N]
    got = M.estimator_from_sums(Nr, joined, CFG["R"])
    ref = O.finalize(CFG["n_levels"] - 1, CFG["R"], True, Nr, want)
    assert got["Q"] == pytest.approx(ref["Q"], rel=1e-15, abs=1e-300)
    assert got["varQ"] == pytest.approx(ref["varQ"], rel=1e-13)
    assert np.allclose(got["Ybar"], ref["Ybar"], rtol=1e-14, atol=0)
    assert np.allclose(got["Vell"], ref["Vell"], rtol=1e-12, atol=0)


def _rank_mixed(rank, world, port, out):
    import torch.distributed as dist

    from oracle import mimc

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    lo, hi = _oracle(mu0=1), _oracle(mu0=2)
    mine = D.shard_work(WORK, CFG["R"], rank, world)
    sums = mimc.mixed_sums(hi, lo, mine)[0] if mine else np.zeros((CFG["n_levels"], CFG["R"], 2))
    t = torch.from_numpy(np.ascontiguousarray(sums).reshape(-1).copy())
    D.allreduce_sums(t)
    if rank == 0:
        np.save(out, t.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_multi_index_sums_equal_single_process():
    # the mixed differences of the multi-index variant shard by shift the same
    # way: every (level, shift) entry comes from the one rank owning the shift,
    # summed over the same samples in the same order, so the join is exact
    import socket

    import torch.multiprocessing as mp

    from oracle import mimc

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = os.path.join(tempfile.mkdtemp(), "mixed.npy")
    mp.start_processes(_rank_mixed, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    joined = np.load(out).reshape(CFG["n_levels"], CFG["R"], 2)
    want, _ = mimc.mixed_sums(_oracle(mu0=2), _oracle(mu0=1), WORK)
    assert np.array_equal(joined, want)
    assert np.any(joined[..., 0] != 0.0)

