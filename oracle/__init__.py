"""FP64 CPU oracle for the resampling F-statistic -- TEST INFRASTRUCTURE ONLY.

A plain, slow, obviously-correct NumPy (float64 / complex128) statement of
what the method computes, written from the paper (Dunn, Clearwater, Melatos &
Wette, "Graphics processing unit implementation of the F-statistic for
continuous gravitational wave searches", arXiv:2201.00451):

* ``geometry``  -- Roemer delay t_m of Sec. 2 (phase model) under a simplified
                   ephemeris, and the antenna patterns a(t), b(t) of Sec. 2
                   (contracted from detector and polarisation tensors).
* ``resamp``    -- the Resamp steps (iii)-(vii) of Sec. 3, one template at a
                   time, following eqs. (Fa), (Fb) and (Fstat) of Sec. 2.
* ``demod``     -- brute-force demodulation: eqs. (Fa_DET), (Fb_DET) summed
                   directly over detector samples (the exact definition).
* ``synth``     -- CW signal injection into seeded noise.
* ``metrics``   -- the comparison metrics r1, r2, theta of Sec. 4.2.
* ``grad``      -- 2F and its gradient in (f, f1dot, alpha, delta) at
                   arbitrary parameters, from the demodulation sums.
* ``peaks``     -- threshold crossings and per-band maxima of 2F (Sec. 5.4,
                   Sec. 4.1).
* ``semicoh``   -- semi-coherent sum of per-segment 2F with nearest-bin
                   sliding (Sec. 6).
* ``interp_study`` -- accuracy of the step-(v) interpolator variants.
* ``sft``       -- step (ii): x_h from short Fourier transforms (Sec. 3).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library and never imports it.
"""

from . import geometry, resamp, demod, synth, metrics, grad, peaks, semicoh, sft  # noqa: F401
