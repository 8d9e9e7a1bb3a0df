"""Denoiser experiment: train the U-Net on pairs the engine generates on
synthetic phantoms, then compare, on held-out phantoms, the wall time plain
Monte Carlo needs to bring every organ dose within 2 % of a high-count
reference with the time Monte Carlo plus the denoiser needs (checkpoints of
low-count decays, each denoised whole-volume).

Everything numerical runs through the C ABI (nm_dose_* for the transport,
nm_denoise_* for the network); this module only orchestrates: phantom
generation on the host (a spawn process pool, started before any GPU work),
device buffers, patch sampling, the training loop and the timing.

    python -m paper_2111_11687_gb300.experiment --train 200 --test 20
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _gen(args):
    from paper_2111_11687_gb300 import inputs
    shape, spacing, seed = args
    ph = inputs.adult_phantom(shape=shape, spacing=spacing, seed=seed)
    return ph.hu, ph.activity, ph.labels, ph.spacing


def make_phantoms(seeds, shape, spacing, workers=None):
    """Adult phantoms for the given seeds, generated in a spawn pool and
    yielded in order (so that the caller can move each to the device and drop
    the host copy)."""
    jobs = [(shape, spacing, s) for s in seeds]
    if workers == 1 or len(jobs) == 1:
        for j in jobs:
            yield _gen(j)
        return
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers or min(len(jobs), os.cpu_count() or 1)) as pool:
        for ph in pool.imap(_gen, jobs, chunksize=1):
            yield ph


class Case:
    """One phantom on the device: density, material, activity, labels."""

    def __init__(self, nm, torch, ph, materials, n_labels, activity_bq):
        hu, act, lab, spacing = ph
        self.shape = hu.shape
        self.spacing = spacing
        self.density = torch.empty(self.shape, dtype=torch.float32, device="cuda")
        self.material = torch.empty(self.shape, dtype=torch.uint8, device="cuda")
        nm.nm_ct_to_phantom(torch.from_numpy(hu).cuda(), self.density, self.material)
        self.activity = torch.from_numpy(act).cuda()
        self.labels = torch.from_numpy(lab).cuda()
        self.nm, self.torch = nm, torch
        self.materials = materials
        self.n_labels = n_labels
        self.activity_bq = activity_bq

    def handle(self, **kw):
        return self.nm.Dose(self.density, self.material, self.spacing, self.materials, activity=self.activity,
                            labels=self.labels, n_labels=self.n_labels, activity_bq=self.activity_bq, **kw)

    def dose(self, n_decays, seed):
        """Dose-rate map (device FP32) after n_decays decays; returns (map, seconds)."""
        out = self.torch.empty(self.shape, dtype=self.torch.float32, device="cuda")
        with self.handle() as d:
            self.torch.cuda.synchronize()
            t0 = time.perf_counter()
            d.run(n_decays, seed)
            self.nm.nm_dose_get(d.h, out, None, None)
            self.torch.cuda.synchronize()
            return out, time.perf_counter() - t0


def body_box(density, margin):
    """Voxel bounding box (z0, z1, y0, y1, x0, x1) of density >= 0.1."""
    idx = (density >= 0.1).nonzero()
    lo = idx.min(0).values.tolist()
    hi = idx.max(0).values.tolist()
    return lo, hi


def train(nm, torch, net, cases, lows, highs, steps, patch, batch, lr, seed, log_every=0):
    rng = np.random.default_rng(seed)
    x = torch.empty((batch, patch, patch, patch, 8), dtype=torch.bfloat16, device="cuda")
    tgt = torch.empty((batch, patch, patch, patch), dtype=torch.float32, device="cuda")
    wgt = torch.empty_like(tgt)
    scales = [nm.nm_denoise_scales(lo, c.activity, c.density) for c, lo in zip(cases, lows)]
    boxes = [body_box(c.density, patch // 2) for c in cases]
    losses = []
    for step in range(steps):
        # one phantom per step, `batch` patch centres drawn inside its body box
        i = int(rng.integers(len(cases)))
        (z0, y0, x0), (z1, y1, x1) = boxes[i]
        corners = np.stack([rng.integers(x0, x1 + 1, batch), rng.integers(y0, y1 + 1, batch),
                            rng.integers(z0, z1 + 1, batch)], 1) - patch // 2
        cd = torch.from_numpy(corners.astype(np.int32)).cuda()
        ds, as_ = scales[i]
        nm.nm_denoise_make_patches(lows[i], cases[i].density, cases[i].activity, highs[i], ds, as_, cd, patch, x,
                                   tgt, wgt)
        lr_t = lr * 0.5 * (1 + np.cos(np.pi * step / steps))
        losses.append(net.train_step(x, tgt, wgt, lr=lr_t))
        if log_every and step % log_every == 0:
            print(f"step {step} loss {losses[-1]:.5f}", flush=True)
    return losses


def validation_loss(nm, torch, net, cases, lows, highs, patch, batch, n_batches=16, seed=11):
    """The training loss (weighted squared error, forward only) of ``net`` on
    fixed patches of held-out phantoms."""
    rng = np.random.default_rng(seed)
    x = torch.empty((batch, patch, patch, patch, 8), dtype=torch.bfloat16, device="cuda")
    tgt = torch.empty((batch, patch, patch, patch), dtype=torch.float32, device="cuda")
    wgt = torch.empty_like(tgt)
    y = torch.empty_like(tgt)
    scales = [nm.nm_denoise_scales(lo, c.activity, c.density) for c, lo in zip(cases, lows)]
    boxes = [body_box(c.density, patch // 2) for c in cases]
    total = 0.0
    for b in range(n_batches):
        i = b % len(cases)
        (z0, y0, x0), (z1, y1, x1) = boxes[i]
        corners = np.stack([rng.integers(x0, x1 + 1, batch), rng.integers(y0, y1 + 1, batch),
                            rng.integers(z0, z1 + 1, batch)], 1) - patch // 2
        cd = torch.from_numpy(corners.astype(np.int32)).cuda()
        ds, as_ = scales[i]
        nm.nm_denoise_make_patches(lows[i], cases[i].density, cases[i].activity, highs[i], ds, as_, cd, patch, x,
                                   tgt, wgt)
        net.forward(x, y)
        total += float((wgt * (y - tgt) ** 2).mean().item())
    return total / n_batches


def organ_error(means, ref, counts, min_voxels=1):
    sel = (counts[1:] >= min_voxels) & (ref[1:] > 0)
    return np.abs(means[1:][sel] / ref[1:][sel] - 1.0)


def time_to_target(case, ref, step_decays, max_decays, target, seed):
    """Plain MC: wall time and decays until every organ is within target of ref."""
    torch = case.torch
    # one batch per checkpoint: the check needs organ means only, and a batch
    # is one transport launch and one fold
    with case.handle(batches=1) as d:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = 0
        while n < max_decays:
            d.run(step_decays, seed)
            n += step_decays
            mean, _, _, cnt = d.organs(eps=False, sigma=False)
            err = organ_error(mean, ref, cnt)
            if err.max() <= target:
                torch.cuda.synchronize()
                return time.perf_counter() - t0, n, float(err.max())
        torch.cuda.synchronize()
        return None, n, float(err.max())


def time_to_target_denoised(case, net, ref, counts, step_decays, max_decays, target, seed, organ_roi=True):
    """MC + denoiser: wall time and decays until the denoised map puts every
    organ within target of ref.  Each checkpoint adds step_decays decays to the
    same run, denoises the whole accumulated map and checks it, so a case the
    network cannot bring within target at the first checkpoint falls back to
    more Monte Carlo.  With organ_roi the network runs on the organs' bounding
    box (the label map) instead of the whole body: only organ doses enter the
    criterion.  Also returns the errors at the first checkpoint."""
    torch, nm = case.torch, case.nm
    raw = torch.empty(case.shape, dtype=torch.float32, device="cuda")
    den = torch.empty_like(raw)
    first = None
    with case.handle(batches=1) as d:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = 0
        while n < max_decays:
            d.run(step_decays, seed)
            n += step_decays
            nm.nm_dose_get(d.h, raw, None, None)
            net.apply(raw, case.density, case.activity, den, roi=case.labels if organ_roi else None)
            err = organ_error(d.map_organs(den), ref, counts)
            if first is None:
                # the undenoised error is for the record only: its time is not counted
                ta = time.perf_counter()
                first = (err, organ_error(d.map_organs(raw), ref, counts), ta - t0)
                t0 += time.perf_counter() - ta
            if err.max() <= target:
                torch.cuda.synchronize()
                return time.perf_counter() - t0, n, float(err.max()), first
        torch.cuda.synchronize()
        return None, n, float(err.max()), first


def run(train_n=200, test_n=20, shape=(300, 256, 256), spacing=(0.2, 0.2, 0.3), low=int(1e7), high=int(1e9),
        ref=int(1e10), denoise_low=int(1e7), steps=10000, patch=64, batch=4, lr=1e-3, workers=None,
        step_decays=int(5e6), max_decays=int(2e9), seed0=1000, log_every=0, candidates=3):
    # the pool is started (first next()) before any GPU work
    phantoms = make_phantoms(list(range(seed0, seed0 + train_n + test_n)), shape, spacing, workers)
    first = next(phantoms)
    import torch

    from paper_2111_11687_gb300 import build, inputs, nmdose as nm
    build.build()
    mats = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    cases = [Case(nm, torch, first, mats, inputs.N_LABELS, inputs.ACTIVITY_BQ)]
    del first
    for ph in phantoms:
        cases.append(Case(nm, torch, ph, mats, inputs.N_LABELS, inputs.ACTIVITY_BQ))
        del ph
    tr, te = cases[:train_n], cases[train_n:]
    t0 = time.perf_counter()
    lows = [c.dose(low, 7)[0] for c in tr]
    highs = [c.dose(high, 8)[0] for c in tr]
    t_data = time.perf_counter() - t0
    # Model selection: `candidates` networks (different initial weights and
    # patch draws) train on the training phantoms but a held-out tenth, and
    # the one with the lowest loss on that tenth is kept.  Training runs
    # differ by which minimum they settle in, and the organ errors follow the
    # loss; the test phantoms play no part in the choice.
    n_val = max(1, train_n // 10) if candidates > 1 else 0
    fit = slice(0, train_n - n_val)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net, losses, val_losses, fit_losses = None, None, [], []
    for k in range(candidates):
        cand = nm.Denoiser(patch=patch, batch=batch, levels=4, base_width=16, seed=1 + k, lr=lr)
        cl = train(nm, torch, cand, tr[fit], lows[fit], highs[fit], steps, patch, batch, lr, seed=5 + k,
                   log_every=log_every)
        v = (validation_loss(nm, torch, cand, tr[train_n - n_val:], lows[train_n - n_val:],
                             highs[train_n - n_val:], patch, batch) if n_val else 0.0)
        val_losses.append(v)
        fit_losses.append(float(np.mean(cl[-50:])))
        if net is None or v < min(val_losses[:-1]):
            if net is not None:
                net.close()
            net, losses = cand, cl
        else:
            cand.close()
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del lows, highs
    results = []
    for j, c in enumerate(te):
        refmap, _ = c.dose(ref, 100 + j)
        with c.handle() as h:
            ref_org = h.map_organs(refmap)
        cnts = np.bincount(c.labels.flatten().cpu().numpy(), minlength=inputs.N_LABELS + 1)
        # plain MC
        t_mc, n_mc, e_mc = time_to_target(c, ref_org, step_decays, max_decays, 0.02, 200 + j)
        # MC + denoiser, checkpoints of denoise_low decays
        t_dn, n_dn, e_dn, (e1_dn, e1_lo, t1) = time_to_target_denoised(c, net, ref_org, cnts, denoise_low,
                                                                       max_decays, 0.02, 300 + j)
        results.append(dict(case=j, plain_mc_s=t_mc, plain_mc_decays=n_mc, plain_mc_err=e_mc,
                            mc_denoiser_s=t_dn, mc_denoiser_decays=n_dn, mc_denoiser_err=e_dn,
                            first_checkpoint_s=t1, denoiser_max_err=float(e1_dn.max()),
                            denoiser_mean_err=float(e1_dn.mean()), low_mc_max_err=float(e1_lo.max()),
                            low_mc_mean_err=float(e1_lo.mean())))
    net.close()
    ok_dn = [r for r in results if r["denoiser_max_err"] <= 0.02]
    med = lambda k: float(np.median([r[k] for r in results if r[k] is not None] or [np.nan]))
    summary = dict(train=train_n, test=test_n, grid=list(shape[::-1]), low=low, high=high, ref=ref,
                   denoise_low=denoise_low, steps=steps, patch=patch, batch=batch, data_s=t_data,
                   train_s=t_train, final_loss=float(np.mean(losses[-50:])), first_loss=float(np.mean(losses[:10])),
                   candidates=candidates, candidate_val_losses=val_losses, candidate_final_losses=fit_losses,
                   plain_mc_s_median=med("plain_mc_s"), mc_denoiser_s_median=med("mc_denoiser_s"),
                   plain_mc_decays_median=med("plain_mc_decays"), mc_denoiser_decays_median=med("mc_denoiser_decays"),
                   denoiser_faster=sum(1 for r in results if r["mc_denoiser_s"] is not None and
                                       (r["plain_mc_s"] is None or r["mc_denoiser_s"] < r["plain_mc_s"])),
                   denoiser_reaches_2pct_first_checkpoint=len(ok_dn), denoiser_max_err_median=float(np.median([r["denoiser_max_err"] for r in results])),
                   low_mc_max_err_median=float(np.median([r["low_mc_max_err"] for r in results])),
                   cases=results)
    return summary


def configs(wb_ref=int(1e10), wb_step=int(5e6), wb_low=int(1e8), seed=1):
    """The workloads other than the adult phantom, measured on one GPU:

    * the 64^3 x 5 mm water cube with a central 0.511 MeV point source (one
      photon per history), decays/s at its 1e6 histories and at 1e8;
    * the 512 x 512 x 600 x (1 x 1 x 3 mm) whole-body phantom with lesions:
      decays/s; plain MC's wall time until all 27 organ means are within 2 %
      of a 1e10-decay reference; and the MC + denoiser arm's cost before any
      check, MC of 1e8 decays plus one inference on the organs' bounding box
      (a network of the configured shape; its time does not depend on the
      weights).  A network is trained only at 2 x 2 x 3 mm here, so that
      cost is the arm's lower bound, not a measured time to 2 %.
    """
    import torch

    from paper_2111_11687_gb300 import build, inputs, nmdose as nm
    build.build()
    out = {}
    # water cube, point source
    cube = inputs.water_cube()
    water = nm.Materials([0.5551], [7.42], inputs.PE_COEFF, inputs.PE_EXP)
    den = torch.from_numpy(cube.density).cuda()
    mat = torch.from_numpy(cube.material).cuda()
    for n in (int(1e6), int(1e8)):
        with nm.Dose(den, mat, cube.spacing, water, source_mode=nm.NM_SOURCE_POINT, point=cube.point) as d:
            d.run(n, seed)                      # first run: autotuning, code loading
            d.reset()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            d.run(n, seed)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            c = d.counters()
        out[f"water_cube_{n:.0e}"] = dict(histories=n, wall_s=wall, decays_per_s_wall=n / wall,
                                          decays_per_s_device=n / (c["transport_ms"] * 1e-3))
    # whole body
    mats = nm.Materials(inputs.MATERIAL_Z_OVER_A, inputs.MATERIAL_ZEFF, inputs.PE_COEFF, inputs.PE_EXP)
    ph = inputs.whole_body_phantom(seed=seed)
    case = Case(nm, torch, (ph.hu, ph.activity, ph.labels, ph.spacing), mats, inputs.N_LABELS,
                inputs.ACTIVITY_BQ)
    del ph
    _, t_1e9 = case.dose(int(1e9), 11)
    refmap, t_ref = case.dose(wb_ref, 12)
    with case.handle() as h:
        ref_org = h.map_organs(refmap)
    del refmap
    t_mc, n_mc, e_mc = time_to_target(case, ref_org, wb_step, int(2e9), 0.02, 13)
    low, t_low = case.dose(wb_low, 14)
    net = nm.Denoiser(patch=64, batch=1, levels=4, base_width=16, seed=1)
    dn = torch.empty_like(low)
    net.apply(low, case.density, case.activity, dn, roi=case.labels)   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.apply(low, case.density, case.activity, dn, roi=case.labels)
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    net.close()
    out["whole_body"] = dict(grid=[512, 512, 600], voxel_mm=[1, 1, 3], decays_per_s_1e9=1e9 / t_1e9,
                             reference_decays=wb_ref, reference_s=t_ref, plain_mc_s=t_mc, plain_mc_decays=n_mc,
                             plain_mc_err=e_mc, mc_low_decays=wb_low, mc_low_s=t_low, inference_s=t_inf,
                             mc_denoiser_lower_bound_s=t_low + t_inf)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=200)
    ap.add_argument("--test", type=int, default=20)
    ap.add_argument("--grid", default="256,256,300")
    ap.add_argument("--voxel-mm", default="2,2,3")
    ap.add_argument("--low", type=float, default=1e7)
    ap.add_argument("--high", type=float, default=1e9)
    ap.add_argument("--ref", type=float, default=1e10)
    ap.add_argument("--denoise-low", type=float, default=1e7)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--patch", type=int, default=64)
    ap.add_argument("--batch", type=int, default=4)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--workers", type=int, default=0)
    ap.add_argument("--log-every", type=int, default=0)
    ap.add_argument("--candidates", type=int, default=3, help="networks trained; the best on held-out phantoms is kept")
    ap.add_argument("--configs", action="store_true", help="measure the water-cube and whole-body workloads instead")
    a = ap.parse_args()
    if a.configs:
        print(json.dumps(configs()))
        return
    nx, ny, nz = (int(v) for v in a.grid.split(","))
    sp = tuple(float(v) / 10 for v in a.voxel_mm.split(","))
    out = run(a.train, a.test, (nz, ny, nx), sp, int(a.low), int(a.high), int(a.ref), int(a.denoise_low), a.steps,
              a.patch, a.batch, a.lr, a.workers or None, log_every=a.log_every, candidates=a.candidates)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
