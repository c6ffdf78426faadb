"""Seeded synthetic workloads: materials, layered geometries, cuts, primaries.

This module holds only input data and seeded random draws of primaries; it
contains none of the transport arithmetic.  Both the CUDA path and the FP64
oracle take their inputs from here.

The workloads stand in for the paper's TestEm5 thin-target and TestEm3
sampling-calorimeter applications (Sec. 4, Fig. "phys1", Tables "phys1" and
"phys2"): a pencil photon beam on a water-like slab, and 50-layer sampling
calorimeters hit by electrons.  Materials are defined by their elements,
mass fractions, density and mean excitation energy (ICRU 37 / NIST values).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

GAMMA, ELECTRON, POSITRON = 0, 1, 2

P_COMPTON, P_PHOTO, P_PAIR, P_BREM, P_IONI, P_ANNIH = (1 << i for i in range(6))
P_ALL = P_COMPTON | P_PHOTO | P_PAIR | P_BREM | P_IONI | P_ANNIH
P_MSC = 1 << 6  # multiple scattering along charged steps (not part of P_ALL)
P_INTEGRAL = 1 << 7  # integral approach for e+- cross sections along a step (not part of P_ALL)

DEFAULT_SEED = 0x6765616E7456  # "geantV"

# primary record, laid out like the C struct of both libraries (natural alignment);
# `id` is the primary's ordinal within its event
PRIMARY_DTYPE = np.dtype(
    [("type", "<i4"), ("E", "<f8"), ("x", "<f8"), ("y", "<f8"), ("z", "<f8"),
     ("u", "<f8"), ("v", "<f8"), ("w", "<f8"), ("event", "<u4"), ("id", "<u4")],
    align=True,
)


@dataclasses.dataclass
class Material:
    name: str
    Z: Sequence[float]
    A: Sequence[float]
    w: Sequence[float]  # mass fractions
    rho: float  # g/cm3
    I_eV: float


@dataclasses.dataclass
class Workload:
    name: str
    materials: List[Material]
    n_layers: int
    sub_thick: Sequence[float]  # cm, per sub-slab of one layer
    sub_mat: Sequence[int]
    half_x: float  # cm, <= 0: unbounded
    half_y: float
    nx: int
    ny: int
    gamma_cut: float  # MeV
    e_cut: float
    track_cut: float
    process_mask: int
    primaries: np.ndarray  # PRIMARY_DTYPE
    n_events: int
    seed: int = DEFAULT_SEED
    field_T: float = 0.0  # uniform magnetic field (tesla) along field_axis (0 x, 1 y, 2 z)
    field_axis: int = 1
    # per final-state model (Compton, pair, brems, Moller, Bhabha, annihilation):
    # rejection sampling at E >= this (MeV) where built, sampling tables below
    reject_min: Optional[Sequence[float]] = None

    @property
    def n_sub(self) -> int:
        return len(self.sub_thick)

    @property
    def n_subtotal(self) -> int:
        return self.n_layers * self.n_sub

    def subset(self, n_events: int) -> "Workload":
        """The first n_events events of this workload (same geometry and seed)."""
        p = self.primaries[self.primaries["event"] < n_events]
        return dataclasses.replace(self, primaries=p.copy(), n_events=n_events,
                                   name=f"{self.name}[:{n_events}]")


# --- materials ---------------------------------------------------------------
# water-like pseudo-element: Z_eff = 7.4 with A chosen so that Z/A is water's 0.55508
WATER_LIKE = Material("water-like", [7.4], [13.331], [1.0], 1.0, 75.0)
LEAD = Material("Pb", [82.0], [207.2], [1.0], 11.35, 823.0)
# polystyrene (C8H8)n: C:H = 1:1 by atoms
_C, _H = 12.011, 1.008
POLYSTYRENE = Material("polystyrene", [6.0, 1.0], [_C, _H],
                       [_C / (_C + _H), _H / (_C + _H)], 1.05, 68.7)
TUNGSTEN = Material("W", [74.0], [183.84], [1.0], 19.3, 727.0)
SILICON = Material("Si", [14.0], [28.0855], [1.0], 2.33, 173.0)
LIQUID_ARGON = Material("LAr", [18.0], [39.948], [1.0], 1.396, 188.0)


def make_primaries(n: int) -> np.ndarray:
    return np.zeros(n, dtype=PRIMARY_DTYPE)


def _pencil(n_events: int, ptype: int, energy: float) -> np.ndarray:
    p = make_primaries(n_events)
    p["type"] = ptype
    p["E"] = energy
    p["w"] = 1.0
    p["event"] = np.arange(n_events, dtype=np.uint32)
    return p


def photon_slab(n_events: int = 100_000, energy: float = 1.0) -> Workload:
    """1 MeV photon pencil beam on a 10 cm water-like slab; Compton +
    photoelectric only; electrons deposited where they are made."""
    return Workload(
        name=f"gamma{energy:g}MeV_water10cm_{n_events}",
        materials=[WATER_LIKE], n_layers=1, sub_thick=[10.0], sub_mat=[0],
        half_x=0.0, half_y=0.0, nx=0, ny=0,
        gamma_cut=1.0, e_cut=1e30, track_cut=1e-3,
        process_mask=P_COMPTON | P_PHOTO,
        primaries=_pencil(n_events, GAMMA, energy), n_events=n_events)


def _pb_ps(name: str, prim: np.ndarray, n_events: int) -> Workload:
    return Workload(
        name=name, materials=[LEAD, POLYSTYRENE], n_layers=50,
        sub_thick=[0.2, 0.5], sub_mat=[0, 1], half_x=20.0, half_y=20.0, nx=0, ny=0,
        gamma_cut=1.0, e_cut=1.0, track_cut=1e-3, process_mask=P_ALL,
        primaries=prim, n_events=n_events)


def pbps_electrons(n_events: int = 1000, energy: float = 1000.0) -> Workload:
    """e- pencil beam on 50 x (2 mm Pb + 5 mm polystyrene), 40x40 cm, cuts 1 MeV."""
    return _pb_ps(f"e-{energy/1000:g}GeV_PbPS50_{n_events}",
                  _pencil(n_events, ELECTRON, energy), n_events)


def pbps_mixed(n_events: int = 4096, seed: int = DEFAULT_SEED) -> Workload:
    """Mixed e-/e+/gamma (1:1:1 by event index), energies log-uniform in
    0.1-100 GeV, on the Pb/polystyrene calorimeter."""
    rng = np.random.default_rng(seed)
    p = _pencil(n_events, GAMMA, 1.0)
    p["type"] = np.arange(n_events) % 3
    p["E"] = 100.0 * 10.0 ** (3.0 * rng.random(n_events))
    w = _pb_ps(f"mixed0.1-100GeV_PbPS50_{n_events}", p, n_events)
    w.seed = seed
    return w


def wsi_cells(n_events: int = 10_000, energy: float = 100_000.0,
              seed: int = DEFAULT_SEED) -> Workload:
    """100 GeV e- on 50 x (3 mm W + 0.5 mm Si) with 32x32 cells of 1.25 cm;
    entry points uniform over the central 4x4 cells; cuts 0.5 MeV."""
    rng = np.random.default_rng(seed + 5)
    p = _pencil(n_events, ELECTRON, energy)
    p["x"] = rng.uniform(-2.5, 2.5, n_events)
    p["y"] = rng.uniform(-2.5, 2.5, n_events)
    return Workload(
        name=f"e-{energy/1000:g}GeV_WSi50_cells_{n_events}",
        materials=[TUNGSTEN, SILICON], n_layers=50, sub_thick=[0.3, 0.05], sub_mat=[0, 1],
        half_x=20.0, half_y=20.0, nx=32, ny=32,
        gamma_cut=0.5, e_cut=0.5, track_cut=1e-3, process_mask=P_ALL,
        primaries=p, n_events=n_events, seed=seed)


def pblar_testem3(n_events: int = 1000, energy: float = 10_000.0) -> Workload:
    """The paper's TestEm3 layout: 50 x (2.3 mm Pb + 5.7 mm LAr), e- beam."""
    return Workload(
        name=f"e-{energy/1000:g}GeV_PbLAr50_{n_events}",
        materials=[LEAD, LIQUID_ARGON], n_layers=50, sub_thick=[0.23, 0.57], sub_mat=[0, 1],
        half_x=20.0, half_y=20.0, nx=0, ny=0, gamma_cut=0.1, e_cut=1.0, track_cut=1e-3,
        process_mask=P_ALL, primaries=_pencil(n_events, ELECTRON, energy), n_events=n_events)


def with_field(wl: Workload, tesla: float = 4.0, axis: int = 1) -> Workload:
    """The same workload in a uniform magnetic field (default: 4 T along y,
    transverse to the beam, as in the paper's TestEm3 set-up)."""
    return dataclasses.replace(wl, field_T=tesla, field_axis=axis, name=f"{wl.name}_B{tesla:g}T{'xyz'[axis]}")


def with_rejection(wl: Workload, reject_min=(0.0, 0.0, 0.0, math.inf, math.inf, math.inf)) -> Workload:
    """The same workload sampling Compton, pair and bremsstrahlung final states
    by rejection above the given energies (MeV), instead of sampling tables."""
    return dataclasses.replace(wl, reject_min=tuple(reject_min), name=wl.name + "_rej")


def with_integral(wl: Workload) -> Workload:
    """The same workload with the integral approach for charged tracks."""
    return dataclasses.replace(wl, process_mask=wl.process_mask | P_INTEGRAL, name=wl.name + "_int")


def with_msc(wl: Workload) -> Workload:
    """The same workload with multiple scattering along charged steps."""
    return dataclasses.replace(wl, process_mask=wl.process_mask | P_MSC, name=wl.name + "_msc")


# The standard workloads, by name.
STANDARD = {
    "gamma1MeV_water10cm_1e5": lambda: photon_slab(100_000, 1.0),
    "e-1GeV_PbPS50_1000": lambda: pbps_electrons(1000, 1000.0),
    "mixed0.1-100GeV_PbPS50_4096": lambda: pbps_mixed(4096),
    "e-10GeV_PbPS50_2000": lambda: pbps_electrons(2000, 10_000.0),
    "e-100GeV_WSi50_cells_1e4": lambda: wsi_cells(10_000, 100_000.0),
}
PHOTON_SLAB, PBPS_1GEV, PBPS_MIXED, PBPS_10GEV, WSI_100GEV = STANDARD


def standard(name: str) -> Workload:
    return STANDARD[name]()
