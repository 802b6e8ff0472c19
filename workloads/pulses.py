"""Sampled incident pulses s(t_n), t_n = n*T/Nt, n = 0..Nt-1 (the signal at the plane d.x = 0).

With the time origin at that plane the incident field is p_inc(x, t) = s(t - d.x/c); the
periodic sampling window of length T makes the train periodic, as in Sec. 4 of the paper.
Units: a = c = 1.
"""
from __future__ import annotations

import numpy as np


def time_grid(Nt: int, T: float) -> np.ndarray:
    return np.arange(Nt, dtype=np.float64) * (T / Nt)


def gaussian_pulse(Nt: int, T: float, sigma: float, tc: float) -> np.ndarray:
    t = time_grid(Nt, T)
    return np.exp(-((t - tc) ** 2) / (2.0 * sigma ** 2))


def ricker_pulse(Nt: int, T: float, kp: float, tc: float) -> np.ndarray:
    """Ricker (Mexican-hat) wavelet whose spectrum peaks at angular frequency kp."""
    t = time_grid(Nt, T)
    a = (kp * (t - tc)) ** 2 / 2.0
    return (1.0 - 2.0 * a) * np.exp(-a)


def modulated_gaussian(Nt: int, T: float, kc: float, sigma: float, tc: float) -> np.ndarray:
    t = time_grid(Nt, T)
    return np.cos(kc * (t - tc)) * np.exp(-((t - tc) ** 2) / (2.0 * sigma ** 2))


def paper_sine_pulse(Nt: int, T: float, k0: float, Nc2: int, alpha: float, t_start: float) -> np.ndarray:
    """The fundamental pulse of Eq. (pulse): sin(tau) exp(-alpha |tau|) for |tau| < pi*Nc2 and zero
    elsewhere, tau = k0 (z - c t) at z = 0, centred at t_start + pi*Nc2/k0 (2N_c = Nc2 cycles)."""
    t = time_grid(Nt, T)
    tau = -k0 * (t - (t_start + np.pi * Nc2 / k0))
    s = np.sin(tau) * np.exp(-alpha * np.abs(tau))
    s[np.abs(tau) >= np.pi * Nc2] = 0.0
    return s
