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


def bulk_rel_l2(a: np.ndarray, b: np.ndarray, drop: float = 1e-3) -> float:
    """Relative L2 of a - b after dropping the `drop` fraction of cells with the largest
    |a - b| (from both norms): the error of the bulk of the field, without the few cells
    where the two precisions took different branches of a discontinuous closure."""
    d = np.abs(a - b).ravel()
    n = int(d.size * drop)
    if n == 0:
        return rel_l2(a, b)
    keep = np.argpartition(d, d.size - n)[: d.size - n]
    return rel_l2(a.ravel()[keep], b.ravel()[keep])


def field_error_table(get_a, get_b, wet_T, T_init=None, S_init=None, fields=STATE):
    """Per-field errors of model a against reference b: relative L2 and max-relative
    (max |a - b| / max |b|) over each field, plus both measures on the tracer anomalies
    T - T_init and S - S_init over the wet cells (the mean of T hides the errors of what
    moved).  get_a, get_b: field name -> array."""
    out = {}
    for f in fields:
        a, b = get_a(f), get_b(f)
        out[f] = {"rel_l2": rel_l2(a, b), "max_rel": max_rel(a, b), "bulk_rel_l2": bulk_rel_l2(a, b)}
        if f in ("T", "S"):
            init = T_init if f == "T" else S_init
            if init is not None:
                da, db = (a - init)[wet_T], (b - init)[wet_T]
                out[f + "_anom"] = {"rel_l2": rel_l2(da, db), "max_rel": max_rel(da, db),
                                    "bulk_rel_l2": bulk_rel_l2(da, db)}
    return out
