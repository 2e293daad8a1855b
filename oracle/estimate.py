"""Noise estimators of Tr(Theta M^{-1}) with subtraction, error bars and relative efficiency.

Test infrastructure (see ``oracle/__init__.py``).

  Tr(Theta M^{-1}) = (1/N) sum_n eta^(n)dag Theta (x^(n) - tilde x^(n)) + Tr(Theta tilde M^{-1})   (Sec. 5)

Sign (Eq. xyz294): <psi-bar Theta psi> = -Tr(Theta M^{-1}); everything here is Tr(Theta M^{-1}).
Error bar (reading; Sec. 7 says "standard error"): sample standard deviation over noises (ddof 1)
of the space-time-summed Re (scalar) or Im (vector) per-noise estimate, divided by sqrt(N).
Relative efficiency (Sec. 7): RE = (1/dy^2 - 1) * 100 with dy = err_method / err_reference.
"""
import numpy as np

from . import operators as O

MODES = ["none", "pert", "poly", "defl", "defl_pert", "defl_poly", "es"]


def noise_terms(U, kappa, etas, ws):
    """Per-noise, per-operator, per-timeslice noise terms eta^dag Theta w: array [n, op, T]."""
    out = []
    for eta, w in zip(etas, ws):
        out.append(O.per_t(O.densities(U, kappa, eta, w)))
    return np.stack(out)


def summarize(per_noise_t, addback_t):
    """per_noise_t: [n, op, T] noise terms; addback_t: [op, T].  Returns dict with
    per-noise totals [n, op], mean [op] (complex), signal [op] (Re or Im of mean),
    stderr [op] of the signal part, and per_t_mean [op, T]."""
    tot = per_noise_t.sum(axis=-1) + addback_t.sum(axis=-1)[None, :]
    n = tot.shape[0]
    mean = tot.mean(axis=0)
    part = np.array([tot[:, i].real if O.OP_PART[i] == 0 else tot[:, i].imag for i in range(O.NOPS)]).T
    signal = part.mean(axis=0)
    err = part.std(axis=0, ddof=1) / np.sqrt(n) if n > 1 else np.full(O.NOPS, np.nan)
    return dict(per_noise=tot, mean=mean, signal=signal, stderr=err,
                per_t_mean=per_noise_t.mean(axis=0) + addback_t)


def relative_efficiency(err_method, err_ref):
    dy = np.asarray(err_method) / np.asarray(err_ref)
    return (1.0 / dy ** 2 - 1.0) * 100.0
