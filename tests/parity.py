"""Helpers comparing the CUDA path with the CPU oracle on the same seeded inputs."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2309_06662_gb300 import ocean

STATE = ["u", "v", "T", "S", "eta"]


def max_rel(a: np.ndarray, b: np.ndarray) -> float:
    """max |a - b| / max |b| (the FP64 parity measure)."""
    scale = np.max(np.abs(b))
    if scale == 0.0:
        return float(np.max(np.abs(a)))
    return float(np.max(np.abs(a - b)) / scale)


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2 (the mixed-precision parity measure)."""
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return float(np.linalg.norm(a))
    return float(np.linalg.norm(a - b) / nb)


def run_pair(case, precision: int, steps: int, params=None):
    m_gpu = ocean.Ocean(case, precision=precision, params=params)
    m_ora = oracle.OracleModel(case, params=params)
    if steps:
        m_gpu.step(steps)
        m_ora.step(steps)
    return m_gpu, m_ora


def state_errors(m_gpu, m_ora, measure=max_rel, fields=STATE):
    return {f: measure(m_gpu.get(f), m_ora.get(f)) for f in fields}
