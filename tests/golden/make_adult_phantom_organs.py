"""Writes adult_phantom_organs_oracle.txt: the FP64 oracle's organ mean dose
rates (paper Eq. 2: the unweighted mean over an organ's voxels of the Eq. 1
dose rate) and the batch standard deviation of each mean, for the benchmark's
adult PET/CT phantom (256x256x300 voxels of 2x2x3 mm, phantom seed 1, 27
organs), from N decays in B batches.  It calls only the oracle and the seeded
input generator, never the CUDA path.

    python tests/golden/make_adult_phantom_organs.py [N] [threads]

N = 1e9 makes the worst organ's relative sigma about 0.27 %, so that against
a 1e10-decay GPU run three combined sigmas stay below the 1 % organ
criterion for all 27 organs."""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2111_11687_gb300 import inputs  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "adult_phantom_organs_oracle.txt")
SHAPE, SPACING, PHANTOM_SEED, SEED, BATCHES = (300, 256, 256), (0.2, 0.2, 0.3), 1, 20211123, 20


def main():
    n = int(float(sys.argv[1])) if len(sys.argv) > 1 else 1_000_000_000
    threads = int(sys.argv[2]) if len(sys.argv) > 2 else 0
    ph = inputs.adult_phantom(shape=SHAPE, spacing=SPACING, seed=PHANTOM_SEED)
    den, mat = oracle.hu_to_phantom(ph.hu)
    om = oracle.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    t0 = time.time()
    r = oracle.run(den, mat, om, activity=ph.activity, labels=ph.labels, n_labels=inputs.N_LABELS, spacing=SPACING,
                   n_hist=n, seed=SEED, batches=BATCHES, threads=threads, activity_bq=inputs.ACTIVITY_BQ)
    dt = time.time() - t0
    cnt = np.bincount(ph.labels.ravel(), minlength=inputs.N_LABELS + 1)
    with open(OUT + ".tmp", "w") as f:
        f.write("# FP64 oracle organ dose rates of the adult PET/CT phantom (paper Eq. 1 and Eq. 2; 18F,\n")
        f.write("# 2 x 0.511 MeV photons + 0.25 MeV local positron energy per decay, A(t_s) of the paper's\n")
        f.write("# patient, §2.2), written by tests/golden/make_adult_phantom_organs.py.\n")
        f.write(f"# grid 256x256x300 voxels of 2x2x3 mm, phantom seed {PHANTOM_SEED}, decays {n}, oracle seed {SEED}, "
                f"batches {BATCHES}, {r.counters['threads_used']} threads, {dt:.0f} s\n")
        f.write("# label mean_Gy_per_s sigma_of_mean_Gy_per_s voxels\n")
        for lab in range(inputs.N_LABELS + 1):
            f.write(f"{lab} {r.organ_mean[lab]:.12e} {r.organ_sigma[lab]:.12e} {cnt[lab]}\n")
    os.replace(OUT + ".tmp", OUT)
    print(f"wrote {OUT}: {n} decays in {dt:.0f} s")


if __name__ == "__main__":
    main()
