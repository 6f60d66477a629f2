"""Semi-coherent sum of per-segment 2F (oracle, test infrastructure).

Sec. 6 describes the search built on this implementation: the data are
split into segments of about ten days, each segment is searched with the
F-statistic, and the segments' results are summed, both on the GPU.  The
sum is stated here by definition, with nearest-bin sliding:

A template (alpha, delta, f1dot, f2dot) has its spindowns at the global
reference time t_ref; global bin m is the frequency f_m = f_h + (m - n/2) df
at t_ref.  Segment s, with its own reference time t_s (offset
D_s = t_s - t_ref), is searched coherently with
    f1dot_s = f1dot + f2dot D_s,   f2dot_s = f2dot,
and the frequency of global bin m at t_s, f_m + f1dot D_s + f2dot D_s^2 / 2,
lies nearest to its bin m + k_s with
    k_s = rint((f1dot D_s + f2dot D_s^2 / 2) / df).
Then
    2F_sum[m] = sum_s 2F_s[m + k_s],
where a term whose bin m + k_s falls outside [0, n) is 0.
"""

from __future__ import annotations

import numpy as np

from . import resamp


def segment_shift(df: float, d_ref: float, f1dot: float, f2dot: float) -> int:
    """k_s: bins by which segment s's frequency axis slides against the global one."""
    return int(np.rint((f1dot * d_ref + 0.5 * f2dot * d_ref * d_ref) / df))


def segment_template(tm, d_ref: float):
    """The segment's coherent template: spindowns carried to its reference time."""
    out = np.array(tm, copy=True)
    out["f1dot"] = tm["f1dot"] + tm["f2dot"] * d_ref
    return out


def semicoherent(segments, data, templates, t_ref: float):
    """2F_sum[n_templates, n_fft] over segment targets (same dt, f_h, n_fft)
    with their x_h lists, for templates with spindowns at t_ref."""
    n_fft = segments[0].n_fft
    df = 1.0 / (n_fft * segments[0].dt)
    out = np.zeros((len(templates), n_fft))
    for seg, x in zip(segments, data):
        d_ref = seg.t_reference - t_ref
        seg_tm = segment_template(templates, d_ref)
        two_f = resamp.fstat(seg, x, seg_tm)
        for i, tm in enumerate(templates):
            k = segment_shift(df, d_ref, float(tm["f1dot"]), float(tm["f2dot"]))
            m = np.arange(n_fft)
            src = m + k
            ok = (src >= 0) & (src < n_fft)
            out[i, ok] += two_f[i, src[ok]]
    return out
