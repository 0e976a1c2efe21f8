"""Helpers shared by the parity tests: run the CUDA path through the C ABI and
the FP64 oracle on the same seeded inputs, and the error metrics the
tolerances are stated in."""
from __future__ import annotations

import numpy as np


def bl_index(n_ant, a, a2):
    return a * n_ant - a * (a - 1) // 2 + (a2 - a)


def vis_norm_error(V, Vref, n_ant, n_pol):
    """max |V - Vref| / sqrt(Vref_aa^pp * Vref_a'a'^qq) over every entry (autos normalise)."""
    nch, nbl, npp = Vref.shape
    autos = np.zeros((nch, n_ant, n_pol))
    for a in range(n_ant):
        b = bl_index(n_ant, a, a)
        for p in range(n_pol):
            autos[:, a, p] = Vref[:, b, p * n_pol + p].real
    worst = 0.0
    b = 0
    for a in range(n_ant):
        for a2 in range(a, n_ant):
            for p in range(n_pol):
                for q in range(n_pol):
                    den = np.sqrt(np.maximum(autos[:, a, p] * autos[:, a2, q], 1e-300))
                    e = np.abs(V[:, b, p * n_pol + q] - Vref[:, b, p * n_pol + q]) / den
                    worst = max(worst, float(e.max()))
            b += 1
    return worst


def vis_self_norm_error(V, Vref, n_ant, n_pol):
    """The same metric for self-polar visibilities [n_chan][n_bl][n_pol] (products pp only)."""
    worst = 0.0
    for a in range(n_ant):
        for a2 in range(a, n_ant):
            b = bl_index(n_ant, a, a2)
            for p in range(n_pol):
                den = np.sqrt(np.maximum(Vref[:, bl_index(n_ant, a, a), p].real *
                                         Vref[:, bl_index(n_ant, a2, a2), p].real, 1e-300))
                worst = max(worst, float((np.abs(V[:, b, p] - Vref[:, b, p]) / den).max()))
    return worst


def beam_errors(B, Bref_inc, Bref_coh, Y, gain, coh_mask, n_pol, beam_avg=1):
    """(incoherent relative error, coherent error normalised by its Cauchy-Schwarz bound)."""
    e_inc = float(np.max(np.abs(B[0] - Bref_inc) / np.maximum(np.abs(Bref_inc), 1e-300)))
    n_ant = len(gain)
    g2 = np.asarray(gain, float) ** 2 * np.asarray(coh_mask, float)
    P = np.zeros(Y.shape[1:])
    for a in range(n_ant):
        if coh_mask[a]:
            for p in range(n_pol):
                P += np.abs(Y[a * n_pol + p]) ** 2
    bound = g2.sum() * P
    if beam_avg > 1:
        bound = bound.reshape(-1, beam_avg, bound.shape[-1]).mean(axis=1)
    e_coh = float(np.max(np.abs(B[1] - Bref_coh) / np.maximum(bound, 1e-300)))
    return e_inc, e_coh
