"""Pins for the oracle's time-domain synthesis (Eqs. an1-an3): on the full
DFT grid it equals numpy's inverse FFT of the same spectrum, and the
synthesised free-field response of the pulse peaks at R/c -/+ Dt with
opposite signs, as Eq. (an1) places it."""
import numpy as np

from oracle import impulse


def test_synthesis_is_the_inverse_fft():
    rng = np.random.default_rng(4)
    nt = 64
    T = 0.05
    df = 1.0 / T
    freqs = df * np.arange(1, nt // 2)          # positive bins below Nyquist
    psi = rng.standard_normal((freqs.size, 3)) + 1j * rng.standard_normal((freqs.size, 3))
    times = np.arange(nt) * T / nt
    p = impulse.synthesize(psi, freqs, df, times, 0.4 * T / nt)
    P = psi * impulse.pulse_spectrum(freqs, 0.4 * T / nt)[:, None]
    spec = np.zeros((nt, 3), np.complex128)
    # with e^{-i omega t}: p_n = sum_m P_m e^{-2 pi i m n / nt} df + c.c. -> conj(ifft(conj)) form
    spec[1:nt // 2] = P
    spec[nt - 1:nt // 2:-1] = np.conj(P)
    ref = np.real(np.fft.fft(spec, axis=0)) * df
    assert np.max(np.abs(p - ref)) < 1e-12 * np.max(np.abs(ref))


def test_free_field_pulse_arrives_at_r_over_c():
    c = 343.0
    T = 0.05
    nt = 512
    df = 1.0 / T
    freqs = df * np.arange(1, nt // 2)
    dt = T / nt
    pulse_dt = 8 * dt
    R = 3.0
    k = 2 * np.pi * freqs / c
    psi = (np.exp(1j * k * R) / (4 * np.pi * R))[:, None]
    times = np.arange(nt) * dt
    p = impulse.synthesize(psi, freqs, df, times, pulse_dt)[:, 0]
    t0 = R / c
    i_max, i_min = int(np.argmax(p)), int(np.argmin(p))
    assert abs(times[i_max] - (t0 + pulse_dt)) <= dt and abs(times[i_min] - (t0 - pulse_dt)) <= dt


def test_wall_model_pairs_printed_in_the_paper():
    """The oracle's reflection coefficient from the admittance reproduces the
    (zeta, R, alpha) pairs the paper prints through Eq. (sp4) (golden file
    with citations), including the sound-hard limit beta = 0."""
    import json
    import os
    from oracle import images
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_wall_models.json")))
    for c in g["cases"]:
        R = complex(images.reflection_from_admittance(1.0 / c["zeta"]))
        assert abs(R - c["R"]) < 1e-12, c
        assert abs((1 - abs(R) ** 2) - c["alpha"]) < 1e-12, c
    h = g["sound_hard"]
    R = complex(images.reflection_from_admittance(h["beta"]))
    assert abs(R - h["R"]) < 1e-15 and abs(1 - abs(R) ** 2 - h["alpha"]) < 1e-15
