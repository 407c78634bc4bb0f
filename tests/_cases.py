"""Shared seeded cases and oracle/GPU layout helpers for the GPU parity tests."""
import functools

import numpy as np

from paper_2103_16073_gb300 import workloads as W


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def maxrel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def seeded_vector(n, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


@functools.lru_cache(maxsize=None)
def workload(name):
    return {
        "small": W.cfg_small,
        "sub": W.cfg_1khz_sub,
        "full": W.cfg_1khz,
        "baffle_sub": W.cfg_baffle_sub,
        # coarse mesh at a high frequency: expansion orders 116 (root children)
        # and 66, above what one shared-memory tile holds
        "high_order": W.cfg_high_order,
        "baffle": W.cfg_baffle,
        "largest": W.cfg_largest,
        # a small room with walls of different admittance and a ragged count
        "ragged": lambda: W.shoebox_workload("ragged-1.3x1.1x0.9-700Hz", 1.3, 1.1, 0.9, (11, 9, 7),
                                             700.0, 0.2, (0.31, 0.42, 0.27), 16, 7,
                                             beta_per_wall=[0.05, 0.5, 0.2 + 0.1j, 0.3, 0.1, 0.25]),
    }[name]()


@functools.lru_cache(maxsize=None)
def oracle_mesh(name):
    from oracle import bem
    wl = workload(name)
    return bem.Mesh(wl.verts, wl.tris)


@functools.lru_cache(maxsize=None)
def oracle_dense(name):
    from oracle import bem
    wl = workload(name)
    m = oracle_mesh(name)
    L, M, LP = bem.dense_operators(m, wl.k)
    A = bem.system_matrix(L, M, wl.k, wl.beta)
    return {"L": L, "M": M, "LP": LP, "A": A}


@functools.lru_cache(maxsize=None)
def oracle_fmm(name, kind, d0=6.0, pmin=12):
    from oracle import fmm
    wl = workload(name)
    return fmm.FMM(oracle_mesh(name), wl.k, wl.beta, kind=kind, d0=d0, pmin=pmin)
