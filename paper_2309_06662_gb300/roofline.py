"""Algorithmic byte counts of the step's kernels (host-side bookkeeping for the roofline).

"Algorithmic" means every field a kernel must read is read once and every field it must
write is written once, per wet cell (3-D kernels) or per wet column (barotropic), at the
storage size `esz` of the path (4 bytes in the mixed form, 8 in FP64).  Neighbour reads
of a stencil are cache hits by construction and are not counted again.

Whole step (the compulsory traffic of the method): read u, v, T, S and the four
tendencies of the previous step, write u, v, T, S and the four new tendencies: 16
words per cell, plus the 2-D barotropic state once per step.
"""
from __future__ import annotations

import hashlib
import json
import os
import re
from typing import Dict, Optional

import numpy as np

STEP_WORDS_PER_CELL = 16

# per wet cell, in words of the path's storage size
KERNEL_WORDS = {
    # reads T, S, u, v; writes w, p, kappa, nu
    "diag": 8,
    # reads T, S, u, v, w, kappa, G_T, G_S; writes G_T, G_S, T, S
    "tracer": 12,
    # reads u, v, w, p, nu, G_u, G_v; writes G_u, G_v, u, v
    "momentum": 11,
    # reads and writes u, v
    "correct": 4,
}


def barotropic_bytes_per_column(esz: int, n_substeps: int, per_pass: int = 6) -> float:
    """Bytes the split-explicit sub-cycle moves per wet column and step, as written: the
    begin kernel (U^n, V^n, H_u, H_v and FP64 eta^n in; U, V, deta, partial sums and the
    eta gradients out, the three accumulators cleared), one temporally blocked pass per
    `per_pass` substeps (state deta, U, V, the six read-only terms and U^n, V^n in; the
    state out and the three accumulators read and written), and the end kernel (the
    accumulators and FP64 eta in, eta and the corrections out).  The accumulators have
    the path's precision (esz bytes: FP32 in the mixed form, FP64 in the FP64 form)."""
    passes = -(-n_substeps // per_pass)
    begin = 12 * esz + 8 + 3 * esz
    one_pass = 14 * esz + 6 * esz
    end = 8 * esz + 16 + 3 * esz
    return begin + passes * one_pass + end


def wet_cells(depth: np.ndarray, z_faces: np.ndarray, min_depth: float) -> int:
    """Number of wet cells under the full-cell rule (centre above the sea floor)."""
    zc = 0.5 * (z_faces[1:] + z_faces[:-1])
    d = np.where(depth >= min_depth, depth, 0.0)
    return int(sum(np.count_nonzero(zc[k] > -d) for k in range(len(zc))))


def wet_columns(depth: np.ndarray, min_depth: float, z_faces: np.ndarray) -> int:
    """Number of wet columns: deep enough and with a wet top level."""
    zc_top = 0.5 * (z_faces[-1] + z_faces[-2])
    return int(np.count_nonzero((depth >= min_depth) & (zc_top > -depth)))


def load_traffic(path: str, workload: str, source_digest: str) -> Optional[Dict[str, float]]:
    """Per-kernel DRAM bytes per wet cell of `workload` from a committed ncu summary
    (lines "traffic_json: {...}"), or None when none matches or the summary was taken on
    a different kernel source (its digest no longer matches)."""
    if not os.path.exists(path):
        return None
    with open(path) as f:
        for line in f:
            if line.startswith("traffic_json:"):
                d = json.loads(line.split(":", 1)[1])
                if d.get("workload") == workload and d.get("source_digest") == source_digest:
                    return d.get("bytes_per_wet_cell")
    return None


def source_digest(csrc: Optional[str] = None) -> str:
    """Digest of the 3-D kernels' source code (comments and layout left out): a traffic
    figure taken on other code is stale.  `csrc`: the source folder (default: this
    package's)."""
    h = hashlib.sha256()
    here = csrc or os.path.join(os.path.dirname(os.path.abspath(__file__)), "csrc")
    for name in ("ocean_kernels.cu", "ocean_internal.cuh"):
        with open(os.path.join(here, name)) as f:
            text = f.read()
        text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)   # block comments
        text = re.sub(r"//[^\n]*", " ", text)                  # line comments
        h.update(" ".join(text.split()).encode())
    return h.hexdigest()[:16]
