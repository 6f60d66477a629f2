"""Run a few templates of a named workload through libfstat, for external
profilers (ncu) and quick checks on a GPU.

    python -m paper_2201_00451_gb300.run_case large --templates 3 --shape 4096,1,2,2,6
    python -m paper_2201_00451_gb300.run_case narrow --templates 16 --fused
    python -m paper_2201_00451_gb300.run_case narrow --templates 3 --peaks
    python -m paper_2201_00451_gb300.run_case narrow --grad 512

Workloads: ``narrow`` = the 10-day two-detector search (1 728 000 samples,
FFT 2^22), ``large`` = the 120-day search (10 368 000 samples, FFT 2^24);
seeded Gaussian noise, the first sky position, the first templates of the
bank.  The templates run twice (the second run is the one to capture, e.g.
``ncu -s <launches of the first> ...``).  ``--shape n1,ca,va,cb,vb`` fixes
the FFT split and CTA shapes (else the autotuner picks), ``--fused`` selects
the persistent launch, ``--peaks`` the on-device reduction (256 band maxima
and 2F > 70 instead of every bin), ``--grad N`` runs fstat_grad for N
off-grid candidates around the first templates instead.
"""

from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import paper_2201_00451_gb300 as pkg
    from workloads import config2, config5, make_noise, template_grid

    ap = argparse.ArgumentParser()
    ap.add_argument("workload", choices=["narrow", "large"])
    ap.add_argument("--templates", type=int, default=4)
    ap.add_argument("--shape", default="")
    ap.add_argument("--fused", action="store_true")
    ap.add_argument("--peaks", action="store_true")
    ap.add_argument("--grad", type=int, default=0)
    args = ap.parse_args(argv)
    pkg.load()
    t = config2() if args.workload == "narrow" else config5()
    xs = [make_noise(t.seed, X, t.n_samples, t.sigmas[X], "c64") for X in range(len(t.detectors))]
    tm = pkg.as_templates(template_grid(t.skies[:1], t.f1dots, t.f2dots))[: args.templates]
    with pkg.FstatPlan.from_target(t) as plan:
        for X in range(len(t.detectors)):
            plan.set_data(X, xs[X], t.sigmas[X])
        if args.shape:
            n1, ca, va, cb, vb = (int(v) for v in args.shape.split(","))
            plan.set_split(n1)
            plan.set_cta(ca, cb, va, vb)
        else:
            plan.autotune()
        plan.set_fused(args.fused)
        if args.grad:
            import numpy as np

            rng = np.random.default_rng(1)
            c = np.zeros(args.grad, dtype=pkg.CANDIDATE_DTYPE)
            c["f"] = t.freq(rng.integers(t.n_fft // 4, 3 * t.n_fft // 4, args.grad))
            c["f1dot"] = tm["f1dot"][rng.integers(0, len(tm), args.grad)]
            c["alpha"], c["delta"] = tm["alpha"][0], tm["delta"][0]
            for _ in range(2):
                twoF, grad = plan.grad(c)
                plan.sync()
            print(f"{args.workload}: {args.grad} candidates, 2F[:4] = {twoF[:4].tolist()}")
            return
        out = torch.empty((len(tm), t.n_fft), dtype=torch.float32, device="cuda")
        for _ in range(2):
            if args.peaks:
                res = plan.compute_peaks(tm, threshold=70.0, n_bands=256, capacity=1 << 16)
            else:
                plan.compute(tm, out=out)
            plan.sync()
        if args.peaks:
            print(f"{args.workload}: {len(tm)} templates (peaks), band maxima[0, :4] = "
                  f"{res['band_max'][0, :4].tolist()}")
        else:
            print(f"{args.workload}: {len(tm)} templates, split {plan.split}, cta {plan.cta}, fused {plan.fused}, "
                  f"2F[0, :4] = {out[0, :4].tolist()}")


if __name__ == "__main__":
    main()
