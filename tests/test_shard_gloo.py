"""The multi-rank path on the CPU: history ranges per rank, the gather of the
ranks' checkpoint images, and the merge, run as two gloo processes.

The ranks' handles are stand-ins built on the oracle (its random numbers are
keyed by the seed and history ids as well), so the merged int64 tally must
equal a single oracle run over all ids bit for bit.
"""
import os
import socket
import tempfile

import numpy as np
import pytest

from paper_2111_11687_gb300 import inputs, shard

SHAPE = (12, 10, 10)
SPACING = (2.0, 2.0, 3.0)
# The oracle seeds its generator per chunk of 1024 histories (keyed by the
# chunk's first id), so a split reproduces the whole run only when every shard
# and batch starts on a chunk boundary: 2 ranks x 2 batches x 1024.  (The GPU
# keys every history, so there any split works.)
N_TOTAL = 4096
SEED = 11


def _problem():
    import oracle
    ph = inputs.adult_phantom(shape=SHAPE, spacing=SPACING, seed=4)
    den, mt = oracle.hu_to_phantom(ph.hu)
    mat = oracle.Materials(z_over_a=inputs.MATERIAL_Z_OVER_A, zeff=inputs.MATERIAL_ZEFF)
    return ph, den, mt, mat


class OracleShard:
    """Stand-in for nmdose.Dose with the calls sharded_run makes; its image
    is [histories, tally...] as int64."""

    def __init__(self):
        self.ph, self.den, self.mt, self.mat = _problem()
        self.next_id = 0
        self.hist = 0
        self.tally = np.zeros(SHAPE, np.int64)

    def seek(self, i):
        self.next_id = int(i)

    def run(self, n, seed):
        import oracle
        if n == 0:
            return
        r = oracle.run(self.den, self.mt, self.mat, activity=self.ph.activity, spacing=SPACING, n_hist=n,
                       seed=seed, batches=2, threads=1, first_history=self.next_id)
        self.tally += r.tally
        self.hist += n
        self.next_id += n

    def checkpoint_size(self):
        return 8 * (1 + self.tally.size)

    def checkpoint(self, out):
        import torch
        img = np.concatenate([[self.hist], self.tally.ravel()]).astype(np.int64)
        out.copy_(torch.from_numpy(img.view(np.uint8)))
        return out

    def merge(self, image):
        arr = image.numpy().view(np.int64)
        self.hist += int(arr[0])
        self.tally += arr[1:].reshape(SHAPE)


def _worker(rank, ws, port, out_dir):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        d = OracleShard()
        is_dst = shard.sharded_run(d, N_TOTAL, SEED, dst=0)
        assert is_dst == (rank == 0)
        first, n = shard.history_range(N_TOTAL, ws, rank)
        np.save(os.path.join(out_dir, f"own{rank}.npy"), np.array([first, n]))
        if is_dst:
            np.save(os.path.join(out_dir, "merged.npy"), d.tally)
            np.save(os.path.join(out_dir, "hist.npy"), np.array([d.hist]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("n,ws", [(0, 1), (1, 2), (7, 2), (3001, 2), (10, 4), (1 << 40, 3)])
def test_history_ranges_partition_the_ids(n, ws):
    ranges = [shard.history_range(n, ws, r) for r in range(ws)]
    first = 0
    for f, c in ranges:
        assert f == first and c >= 0
        first += c
    assert first == n
    counts = [c for _, c in ranges]
    assert max(counts) - min(counts) <= 1
    with pytest.raises(ValueError):
        shard.history_range(n, ws, ws)


def test_two_gloo_ranks_merge_to_the_single_run(orc):
    import torch.multiprocessing as mp
    ws = 2
    with tempfile.TemporaryDirectory() as out_dir:
        mp.start_processes(_worker, args=(ws, _free_port(), out_dir), nprocs=ws, join=True, start_method="spawn")
        merged = np.load(os.path.join(out_dir, "merged.npy"))
        hist = int(np.load(os.path.join(out_dir, "hist.npy"))[0])
        own = [tuple(np.load(os.path.join(out_dir, f"own{r}.npy"))) for r in range(ws)]
    assert own == [(0, 2048), (2048, 2048)]
    assert hist == N_TOTAL
    ph, den, mt, mat = _problem()
    whole = orc.run(den, mt, mat, activity=ph.activity, spacing=SPACING, n_hist=N_TOTAL, seed=SEED, batches=2,
                    threads=1)
    np.testing.assert_array_equal(merged, whole.tally)
    assert merged.sum() > 0
