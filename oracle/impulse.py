"""Time-domain synthesis of a room response from frequency-domain solutions
(Sec. 4, Eqs. an1-an3) -- oracle, test infrastructure.

Time convention e^{-i omega t}: a real signal p(t) with spectrum
P(omega) = int p(t) e^{i omega t} dt is p(t) = (1/2 pi) int P e^{-i omega t} d omega
= 2 Re int_0^inf P(f) e^{-i 2 pi f t} df; sampled on the frequencies
f_m = m df (m = 1..nf, no f = 0 term) it becomes
    p(t) = 2 df Re sum_m P(f_m) e^{-i 2 pi f_m t}.
The source signal of Eq. (an3), f(t) = delta(t - Dt) - delta(t + Dt), has
F(omega) = e^{i omega Dt} - e^{-i omega Dt} = 2 i sin(omega Dt), and the
response at a receiver is P = psi F with psi the Helmholtz solution for a
unit monopole (G = e^{ikR}/(4 pi R) for the free field), so each image of
Eq. (an1) contributes A_j f(t - R_j/c) / (4 pi R_j).
"""
from __future__ import annotations

import numpy as np


def pulse_spectrum(freqs, pulse_dt):
    """F(omega) of Eq. (an3) at the frequencies (Hz)."""
    return 2j * np.sin(2 * np.pi * np.asarray(freqs) * pulse_dt)


def synthesize(psi, freqs, df, times, pulse_dt):
    """p[t, r] = 2 df Re sum_m psi[m, r] F(f_m) e^{-i 2 pi f_m t}."""
    psi = np.asarray(psi)
    F = pulse_spectrum(freqs, pulse_dt)
    out = np.zeros((len(times), psi.shape[1]))
    for n, t in enumerate(times):
        ph = np.exp(-2j * np.pi * np.asarray(freqs) * t)
        out[n] = 2 * df * np.real(np.sum((psi * (F * ph)[:, None]), axis=0))
    return out
