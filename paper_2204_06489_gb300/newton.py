"""Gauss-Newton drivers over the C ABI (Sec. 3 and Sec. 6).

``newton(fwi, opts, steps)`` runs full Gauss-Newton steps s <- s + ds (no line
search) at the context's frequencies.  ``frequency_continuation`` follows the
paper's second experiment: frequencies from low to high, a fixed number of
Gauss-Newton steps per frequency, the updated model passed on to the next
frequency (one context per frequency; each keeps its own absorbing layer frozen
at the starting model).
"""
from __future__ import annotations

from dataclasses import replace
from typing import Callable, List, Sequence

import numpy as np

from .api import FWI, Opts, default_opts


def newton(fwi: FWI, opts: Opts | None = None, steps: int = 1, inst: int = 0) -> List[dict]:
    opts = opts if opts is not None else default_opts()
    hist = []
    for _ in range(steps):
        ds, st = fwi.newton_step(opts)
        st["ds_norm"] = float(np.linalg.norm(ds))
        hist.append(st)
    return hist


def frequency_continuation(grid, survey, gamma0: np.ndarray, observed: Callable[[float], np.ndarray],
                           freqs: Sequence[float], steps_per_freq: int = 1, opts: Opts | None = None,
                           eps_schedule: Sequence[float] | None = None, stream=None):
    """Run ``steps_per_freq`` Gauss-Newton steps per frequency, low to high.

    ``observed(f)`` returns the data [1, rec_total] of frequency f.  Returns
    (final model [nz, nx], per-step stats with the frequency and misfits)."""
    opts = opts if opts is not None else default_opts()
    gamma = np.array(gamma0, dtype=np.float64)
    gamma_ref = float(np.mean(gamma0))
    layer_model = np.array(gamma0, dtype=np.float64)
    log = []
    for k, f in enumerate(sorted(freqs)):
        o = Opts.from_buffer_copy(opts)
        if eps_schedule is not None:
            o.eps = float(eps_schedule[k])
        sv = replace(survey, freqs_hz=[float(f)])
        ctx = FWI([grid], stream)
        ctx.set_survey(0, sv)
        ctx.set_model(0, layer_model, gamma_ref)     # freezes the layer at the starting model
        ctx.set_model(0, gamma, gamma_ref)
        ctx.set_observed(0, observed(f))
        for _ in range(steps_per_freq):
            _, mis0, _ = ctx.forward(o, want_data=False)
            ds, st = ctx.newton_step(o)
            st.update(freq_hz=float(f), misfit_before=float(mis0[0]))
            log.append(st)
        gamma = ctx.get_model(0)
        _, mis1, _ = ctx.forward(o, want_data=False)
        log[-1]["misfit_after"] = float(mis1[0])
        ctx.close()
    return gamma, log
