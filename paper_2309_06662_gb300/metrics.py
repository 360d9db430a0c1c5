"""Throughput measures of the ocean step (host-side arithmetic only)."""
from __future__ import annotations

SECONDS_PER_DAY = 86400.0
DAYS_PER_YEAR = 365.0


def sim_days_per_day(dt: float, seconds_per_step: float) -> float:
    """Simulated days per wall-clock day: dt / t_step."""
    return dt / seconds_per_step


def sypd(dt: float, seconds_per_step: float) -> float:
    """Simulated years per wall-clock day, dt / (t_step * 365) (the paper's SYPD)."""
    return sim_days_per_day(dt, seconds_per_step) / DAYS_PER_YEAR


def cell_updates_per_s(nx: int, ny: int, nz: int, seconds_per_step: float, steps: int = 1,
                       replicas: int = 1) -> float:
    """Grid cells (land included, as the paper counts grid size) advanced per second."""
    return float(nx) * ny * nz * steps * replicas / seconds_per_step
