"""RowSel sharded by NTT point across ranks (paper Sec. 6, database sharding):
the partition and the reassembly, tested with world_size 2 on the CPU (gloo).

Each rank takes its slot range of the database and of the selection
ciphertexts, computes its part of the output with the oracle (the GPU path is
a RowSel on the same compact slices: a ring of T = N / W points), the ranks
all-gather their slices and reassemble; the result must equal the oracle on
the whole problem. No GPU is used here."""

import os
import socket

import numpy as np
import pytest

import oracle
import synth
from paper_2604_04696_gb300 import shard


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, result_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        primes = synth.PRIMES_28
        B, D0, D1, L, N = 3, 20, 7, 2, 64
        ct = synth.ct_tensor(71, B, D0, L, N, primes)
        db = synth.db_tensor(71, D0, D1, L, N, primes)
        sh = shard.SlotShard(N, world, rank)
        part = oracle.rowsel(sh.take(ct), sh.take(db), list(primes))      # [B][D1][2][L][T]
        full = shard.gather(torch.from_numpy(part.view(np.int32)))
        got = full.numpy().view(np.uint32)
        ok = bool(np.array_equal(got, oracle.rowsel(ct, db, list(primes))))
        with open(result_path + ".%d" % rank, "w") as fh:
            fh.write("ok" if ok else "mismatch")
    finally:
        dist.destroy_process_group()


def test_slot_shards_reassemble_to_the_whole_rowsel(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    path = str(tmp_path / "res")
    mp.start_processes(_rank_main, args=(world, _free_port(), path), nprocs=world, start_method="spawn", join=True)
    for r in range(world):
        with open(path + ".%d" % r) as fh:
            assert fh.read() == "ok", r


def test_shard_plan():
    s = shard.SlotShard(4096, 4, 3)
    assert (s.t0, s.t1, s.T) == (3072, 4096, 1024)
    x = np.arange(2 * 4096).reshape(2, 4096)
    assert np.array_equal(shard.assemble([shard.SlotShard(4096, 4, r).take(x) for r in range(4)]), x)
    for bad in [(4096, 3, 0), (4096, 2, 2), (96, 2, 0)]:
        with pytest.raises(ValueError):
            shard.SlotShard(*bad)


def test_shard_is_a_valid_parameter_set():
    """A shard of T = N / W points with the full ring's primes passes the
    library's parameter checks (q = 1 mod 2N implies q = 1 mod 2T)."""
    from paper_2604_04696_gb300 import _build
    _build.build()
    from paper_2604_04696_gb300 import gpir as g
    for world in (1, 2, 4, 8):
        p = g.gpir_params_create(4096 // world, list(synth.PRIMES_28))
        g.gpir_params_destroy(p)
