"""The run's exchange step with real checkpoint images: two processes (one
gloo rank each, both on the one GPU of this run, whose kernels never wait on
each other) simulate disjoint history ranges with the library, write their
statistics with nm_dose_checkpoint, gather the images over gloo and merge them
with nm_dose_merge on rank 0.  The merged tally, dose map and counters must
equal, bit for bit, one handle that ran every history."""
import json
import os
import socket
import tempfile

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPE = (30, 26, 26)
SPACING = (1.97, 1.97, 3.0)
N_TOTAL = 3_000_001          # odd: the ranks' shares differ by one history
SEED = 17


def _handle(nm):
    from paper_2111_11687_gb300 import inputs
    ph = inputs.adult_phantom(shape=SHAPE, spacing=SPACING, seed=11)
    den = np.empty(ph.shape, np.float32)
    mat = np.empty(ph.shape, np.uint8)
    nm.nm_ct_to_phantom(ph.hu, den, mat)
    gm = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    return nm.Dose(den, mat, ph.spacing, gm, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS,
                   batches=4)


def _rank(rank, port, out_dir):
    import torch.distributed as dist

    from paper_2111_11687_gb300 import nmdose as nm, shard
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=2)
    nm.load()
    with _handle(nm) as d:
        merged = shard.sharded_run(d, N_TOTAL, SEED)
        if merged:
            np.save(os.path.join(out_dir, "tally.npy"), d.tally())
            dose = np.empty(SHAPE, np.float32)
            nm.nm_dose_get(d.h, dose, None, None)
            np.save(os.path.join(out_dir, "dose.npy"), dose)
            json.dump(d.counters(), open(os.path.join(out_dir, "counters.json"), "w"))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_merge_real_checkpoint_images():
    import torch.multiprocessing as mp

    from paper_2111_11687_gb300 import build, nmdose as nm
    build.build()
    nm.load()
    with tempfile.TemporaryDirectory() as tmp:
        mp.start_processes(_rank, args=(_free_port(), tmp), nprocs=2, join=True, start_method="spawn")
        tally = np.load(os.path.join(tmp, "tally.npy"))
        dose = np.load(os.path.join(tmp, "dose.npy"))
        c = json.load(open(os.path.join(tmp, "counters.json")))
    with _handle(nm) as d:
        d.run(N_TOTAL, SEED)
        ref_t = d.tally()
        ref_d = np.empty(SHAPE, np.float32)
        nm.nm_dose_get(d.h, ref_d, None, None)
        rc = d.counters()
    assert np.array_equal(tally, ref_t)
    assert np.array_equal(dose, ref_d)
    for k in ("histories", "emitted", "deposited", "escaped", "killed", "steps", "compton", "photo", "escapes"):
        assert c[k] == rc[k], k
    assert c["batches"] == 2 * rc["batches"]      # each rank's batches are batches of the merged run
