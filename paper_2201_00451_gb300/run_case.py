"""Run a few templates of a named workload through libfstat, for external
profilers (ncu) and quick checks on a GPU.

    python -m paper_2201_00451_gb300.run_case large --templates 3 --shape 4096,1,2,2,6
    python -m paper_2201_00451_gb300.run_case narrow --templates 16 --fused

Workloads: ``narrow`` = the 10-day two-detector search (1 728 000 samples,
FFT 2^22), ``large`` = the 120-day search (10 368 000 samples, FFT 2^24);
seeded Gaussian noise, the first sky position, the first templates of the
bank.  The templates run twice (the second run is the one to capture, e.g.
``ncu -s <launches of the first> ...``).  ``--shape n1,ca,va,cb,vb`` fixes
the FFT split and CTA shapes (else the autotuner picks), ``--fused`` selects
the persistent launch.
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
        out = torch.empty((len(tm), t.n_fft), dtype=torch.float32, device="cuda")
        for _ in range(2):
            plan.compute(tm, out=out)
            plan.sync()
        print(f"{args.workload}: {len(tm)} templates, split {plan.split}, cta {plan.cta}, fused {plan.fused}, "
              f"2F[0, :4] = {out[0, :4].tolist()}")


if __name__ == "__main__":
    main()
