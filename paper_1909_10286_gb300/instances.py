"""Seeded synthetic instances of the biomass-logistics problem.

This module only draws instance data. It holds none of the search method:
no distances, no decoding, no scoring, no local minimisation. Both the CUDA
path and the CPU oracle consume what it returns, so neither depends on the
other for its inputs.

The recipes follow the paper's experimental setup (Sec. 3.1): the HQ sits at
the origin, fields and BPs are uniform in a square centred on it, field sizes
are uniform, the expected supply of a field is yield x area (Eq. 3), and every
BP has the same minimum demand. The fleet tables are per unit: each HU has its
own working rate and each SU its own capacity, speed and fill area, which
generalises Table 1's one HU class and two SU classes.

Every array is float32, so both consumers see identical FP32 inputs.

The field-size, fleet and demand distributions per workload:

* ``tiny``: 6 fields, 2 BPs, 20 x 20 km, area U[5,50] ha, yield 40 t/ha,
  2 tours, 3 HUs (U[1.5,3] ha/h), 4 SUs (U[20,30] t), all speeds 40 km/h,
  demand 80 % of supply.
* ``paper``: 40 fields, 5 BPs, 50 x 50 km, area U[5,80] ha, yield N(40,5) t/ha,
  3 tours, 10 HUs (U[1.5,4] ha/h), 20 SUs (U[18,32] t, U[30,50] km/h),
  HU road speed 40 km/h, demand 90 % of supply.
* ``batched``: sizes per instance fields U{10..120}, BPs U{2..10},
  tours U{1..6}, HUs U{2..20}, SUs U{4..40} (HU and SU counts raised to at
  least the tour count), otherwise as ``paper``.
* ``large``: 300 fields, 20 BPs, 150 x 150 km, 10 tours, 60 HUs, 120 SUs,
  otherwise as ``paper``.
* ``replica``: Table 1 and Sec. 3.1 values: 1200 fields of 3+4u ha, 20 BPs of
  250 ha demand, 80 x 80 km, 7 tours, 7 HUs at 2.5 ha/h, 14 small and 28 large
  SUs. Supply is expressed in hectares as in Sec. 3.1, so capacities are
  converted with the conversion parameter of 40 t/ha.

The SU fill area (hectares harvested while one SU fills up) is the capacity
divided by the instance's mean yield. For the replica it is the Table 1 fill
time times the HU working rate.
"""
from __future__ import annotations

import dataclasses

import numpy as np

F32 = np.float32


@dataclasses.dataclass
class Instance:
    """One problem instance. Node 0 is the HQ, nodes 1..B the BPs, B+1.. the fields."""

    n_fields: int
    n_bps: int
    n_tours: int
    n_hu: int
    n_su: int
    xy: np.ndarray            # (1+B+F, 2) km
    area_ha: np.ndarray       # (F,)
    supply_t: np.ndarray      # (F,)
    demand_t: np.ndarray      # (B,)
    hu_rate_ha_h: np.ndarray  # (H,)
    hu_speed_kmh: float
    su_cap_t: np.ndarray      # (S,)
    su_fill_ha: np.ndarray    # (S,)
    su_speed_kmh: np.ndarray  # (S,)
    name: str = ""
    seed: int = 0
    dist: np.ndarray | None = None   # optional (N, N) km; None = straight lines from xy

    @property
    def n_nodes(self) -> int:
        return 1 + self.n_bps + self.n_fields


WORKLOADS = ("tiny", "paper", "batched", "large", "replica")

# search settings that accompany each workload: (candidates per iteration, iterations)
SEARCH = {
    "tiny": (1 << 14, 50),
    "paper": (1 << 20, 1000),
    "batched": (1 << 16, 500),
    "large": (1 << 24, 2000),
    "replica": (1 << 20, 5000),
}


def _finish(name, seed, rng, F, B, T, H, S, half, area, yld, hu_lo, hu_hi,
            cap_lo, cap_hi, su_v_lo, su_v_hi, hu_speed, rho) -> Instance:
    xy = np.zeros((1 + B + F, 2), dtype=F32)
    xy[1:] = rng.uniform(-half, half, size=(B + F, 2)).astype(F32)
    area = area.astype(F32)
    supply = (yld.astype(F32) * area).astype(F32)
    demand = np.full(B, rho * float(supply.astype(np.float64).sum()) / B, dtype=F32)
    hu_rate = rng.uniform(hu_lo, hu_hi, size=H).astype(F32)
    su_cap = rng.uniform(cap_lo, cap_hi, size=S).astype(F32)
    if su_v_lo == su_v_hi:
        su_speed = np.full(S, su_v_lo, dtype=F32)
    else:
        su_speed = rng.uniform(su_v_lo, su_v_hi, size=S).astype(F32)
    mean_yield = float(supply.astype(np.float64).sum() / area.astype(np.float64).sum())
    su_fill = (su_cap.astype(np.float64) / mean_yield).astype(F32)
    return Instance(F, B, T, H, S, xy, area, supply, demand, hu_rate, float(F32(hu_speed)),
                    su_cap, su_fill, su_speed, name=name, seed=seed)


def make_instance(workload: str, seed: int = 0) -> Instance:
    """Draw one instance of the named workload from a seeded generator."""
    rng = np.random.default_rng([0xB10, seed, WORKLOADS.index(workload)])
    if workload == "tiny":
        F, B, T, H, S = 6, 2, 2, 3, 4
        area = rng.uniform(5.0, 50.0, size=F)
        return _finish(workload, seed, rng, F, B, T, H, S, 10.0, area, np.full(F, 40.0),
                       1.5, 3.0, 20.0, 30.0, 40.0, 40.0, 40.0, 0.8)
    if workload in ("paper", "large"):
        if workload == "paper":
            F, B, T, H, S, half = 40, 5, 3, 10, 20, 25.0
        else:
            F, B, T, H, S, half = 300, 20, 10, 60, 120, 75.0
        area = rng.uniform(5.0, 80.0, size=F)
        yld = np.clip(rng.normal(40.0, 5.0, size=F), 1.0, None)
        return _finish(workload, seed, rng, F, B, T, H, S, half, area, yld,
                       1.5, 4.0, 18.0, 32.0, 30.0, 50.0, 40.0, 0.9)
    if workload == "batched":
        F = int(rng.integers(10, 121))
        B = int(rng.integers(2, 11))
        T = int(rng.integers(1, 7))
        H = max(int(rng.integers(2, 21)), T)
        S = max(int(rng.integers(4, 41)), T)
        area = rng.uniform(5.0, 80.0, size=F)
        yld = np.clip(rng.normal(40.0, 5.0, size=F), 1.0, None)
        return _finish(workload, seed, rng, F, B, T, H, S, 25.0, area, yld,
                       1.5, 4.0, 18.0, 32.0, 30.0, 50.0, 40.0, 0.9)
    if workload == "replica":
        F, B, T, H = 1200, 20, 7, 7
        n_small, n_large = 14, 28
        S = n_small + n_large
        xy = np.zeros((1 + B + F, 2), dtype=F32)
        xy[1:] = rng.uniform(-40.0, 40.0, size=(B + F, 2)).astype(F32)
        area = (3.0 + 4.0 * rng.uniform(0.0, 1.0, size=F)).astype(F32)
        supply = area.copy()                      # Sec. 3.1: supply expressed in ha
        demand = np.full(B, 250.0, dtype=F32)
        hu_rate = np.full(H, 2.5, dtype=F32)
        conv = 40.0                               # t/ha (Table 1)
        su_cap = np.array([12.5 / conv] * n_small + [16.5 / conv] * n_large, dtype=F32)
        su_fill = np.array([6.0 / 60.0 * 2.5] * n_small + [8.0 / 60.0 * 2.5] * n_large, dtype=F32)
        su_speed = np.full(S, 40.0, dtype=F32)
        return Instance(F, B, T, H, S, xy, area, supply, demand, hu_rate, 40.0,
                        su_cap, su_fill, su_speed, name=workload, seed=seed)
    raise ValueError(f"unknown workload {workload!r}")


def make_sized(F: int, B: int, T: int, H: int, S: int, seed: int = 0) -> Instance:
    """An instance with the paper workload's value distributions at chosen sizes
    (edge cases: instances near a kernel shape's limits)."""
    rng = np.random.default_rng([0xB11, seed, F, B, T, H, S])
    half = 25.0 * float(np.sqrt(F / 40.0))   # field density of the paper workload
    area = rng.uniform(5.0, 80.0, size=F)
    yld = np.clip(rng.normal(40.0, 5.0, size=F), 1.0, None)
    return _finish(f"sized{F}x{B}x{T}x{H}x{S}", seed, rng, F, B, T, H, S, half, area, yld,
                   1.5, 4.0, 18.0, 32.0, 30.0, 50.0, 40.0, 0.9)


def make_batch(workload: str, seeds) -> list[Instance]:
    return [make_instance(workload, int(s)) for s in seeds]


def custom_instance(xy, area, supply, demand, hu_rate, hu_speed, su_cap, su_fill, su_speed,
                    n_tours: int, name: str = "custom", dist=None) -> Instance:
    """Wrap hand-written arrays (test fixtures) as an Instance, rounding to float32."""
    xy = np.asarray(xy, dtype=F32).reshape(-1, 2)
    area = np.asarray(area, dtype=F32)
    B = len(demand)
    F = len(area)
    assert xy.shape[0] == 1 + B + F
    return Instance(F, B, int(n_tours), len(hu_rate), len(su_cap), xy, area,
                    np.asarray(supply, dtype=F32), np.asarray(demand, dtype=F32),
                    np.asarray(hu_rate, dtype=F32), float(F32(hu_speed)),
                    np.asarray(su_cap, dtype=F32), np.asarray(su_fill, dtype=F32),
                    np.asarray(su_speed, dtype=F32), name=name,
                    dist=None if dist is None else np.asarray(dist, dtype=F32))
