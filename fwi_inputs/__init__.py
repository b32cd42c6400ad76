"""Seeded synthetic inputs shared by the CUDA path, the benchmarks and the oracle.

This module only *describes* problems: grid sizes, velocity models, source and
receiver positions, frequencies.  It holds none of the method's arithmetic (no
PML, no operator, no solver); both the CUDA library and the CPU oracle take its
outputs as plain arrays.

The paper's experiments use a part of the Marmousi model (Sec. 6), which is not
available here; the layered-and-faulted generator below is a seeded stand-in of
the same character (water layer, dipping sediments, normal faults, 1.5-4.7 km/s).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence

import numpy as np
from scipy.ndimage import gaussian_filter


@dataclass(frozen=True)
class Grid:
    """A 2D survey grid: ``nx`` x ``nz`` core nodes at spacing ``h`` metres,
    ``npml`` absorbing-layer nodes on each of the four sides.  ``pml_c`` is the
    reference velocity (m/s) that sets the absorbing-layer strength and
    ``pml_R`` its target reflection coefficient."""

    nx: int
    nz: int
    npml: int
    h: float
    pml_c: float = 3000.0
    pml_R: float = 1e-3


@dataclass
class Survey:
    """Sources and receivers of one instance, in core-node indices (x fast)."""

    freqs_hz: List[float]
    src_ix: np.ndarray          # int32 [n_src]
    src_iz: np.ndarray          # int32 [n_src]
    src_amp: np.ndarray         # complex128 [n_src]
    rec_offsets: np.ndarray     # int32 [n_src + 1], CSR offsets into rec_ix/rec_iz
    rec_ix: np.ndarray          # int32 [n_rec_total]
    rec_iz: np.ndarray          # int32 [n_rec_total]
    rec_w: np.ndarray           # float64 [n_rec_total], data weights W (diagonal)

    @property
    def n_src(self) -> int:
        return int(self.src_ix.shape[0])

    @property
    def n_freq(self) -> int:
        return len(self.freqs_hz)


def surface_survey(nx: int, n_src: int, freqs_hz: Sequence[float], depth: int = 2,
                   rec_every: int = 1) -> Survey:
    """``n_src`` unit point sources evenly spaced at core depth ``depth``, source
    k at column round((k+1)(nx-1)/(n_src+1)); receivers at every ``rec_every``-th
    core column at the same depth, shared by all sources, weight 1."""
    src_ix = np.array([int(round((k + 1) * (nx - 1) / (n_src + 1))) for k in range(n_src)],
                      dtype=np.int32)
    src_iz = np.full(n_src, depth, dtype=np.int32)
    cols = np.arange(0, nx, rec_every, dtype=np.int32)
    rec_ix = np.tile(cols, n_src).astype(np.int32)
    rec_iz = np.full(rec_ix.shape, depth, dtype=np.int32)
    rec_offsets = (np.arange(n_src + 1) * cols.size).astype(np.int32)
    return Survey(freqs_hz=list(map(float, freqs_hz)), src_ix=src_ix, src_iz=src_iz,
                  src_amp=np.ones(n_src, dtype=np.complex128), rec_offsets=rec_offsets,
                  rec_ix=rec_ix, rec_iz=rec_iz, rec_w=np.ones(rec_ix.shape, dtype=np.float64))


# ----------------------------------------------------------------------------
# velocity models (m/s on the core grid, array [nz, nx], x fast)
# ----------------------------------------------------------------------------

def gradient_anomaly_model(nx: int, nz: int, seed: int = 0, v_top: float = 1500.0,
                           v_bottom: float = 3000.0, dv: float = 300.0,
                           sigma_cells: float = 5.0) -> np.ndarray:
    """Velocity rising linearly with depth from ``v_top`` to ``v_bottom`` plus one
    Gaussian anomaly (+``dv``, std ``sigma_cells``) centred at a seeded random
    core node."""
    rng = np.random.default_rng(seed)
    z = np.arange(nz, dtype=np.float64)[:, None]
    x = np.arange(nx, dtype=np.float64)[None, :]
    v = v_top + (v_bottom - v_top) * z / max(nz - 1, 1) + 0.0 * x
    cx = rng.uniform(0, nx - 1)
    cz = rng.uniform(0, nz - 1)
    v = v + dv * np.exp(-((x - cx) ** 2 + (z - cz) ** 2) / (2.0 * sigma_cells ** 2))
    return v


def layered_faulted_model(nx: int, nz: int, h: float, seed: int = 0, n_layers: int = 30,
                          n_faults: int = 3, v_water: float = 1500.0, v_min: float = 1700.0,
                          v_max: float = 4700.0) -> np.ndarray:
    """Seeded stand-in for a Marmousi-like section: a flat water layer (thickness
    8-12 % of the depth), ``n_layers`` dipping interfaces (dips within +-8 deg)
    with velocities increasing with layer index from ``v_min`` to ``v_max``
    (+-75 m/s jitter, kept monotone), cut by ``n_faults`` normal faults dipping
    60 deg with 40-160 m throws (hanging wall down)."""
    rng = np.random.default_rng(seed)
    depth = (nz - 1) * h
    width = (nx - 1) * h
    z_w = rng.uniform(0.08, 0.12) * depth
    z0 = np.sort(rng.uniform(z_w, depth, size=n_layers))
    dips = np.deg2rad(rng.uniform(-8.0, 8.0, size=n_layers))
    v_lay = np.linspace(v_min, v_max, n_layers + 1) + rng.uniform(-75.0, 75.0, size=n_layers + 1)
    v_lay = np.maximum.accumulate(v_lay)
    f_x = rng.uniform(0.15 * width, 0.85 * width, size=n_faults)
    f_throw = rng.uniform(40.0, 160.0, size=n_faults)
    f_sign = rng.choice([-1.0, 1.0], size=n_faults)
    t60 = np.tan(np.deg2rad(60.0))

    z = (np.arange(nz, dtype=np.float64) * h)[:, None]
    x = (np.arange(nx, dtype=np.float64) * h)[None, :]
    z_eff = np.broadcast_to(z, (nz, nx)).copy()
    for k in range(n_faults):
        # fault plane x = f_x + sign * (z - z_w) / tan(60); hanging wall on the dip side
        plane = f_x[k] + f_sign[k] * (z - z_w) / t60
        hanging = (f_sign[k] * (x - plane) > 0) & (z > z_w)
        z_eff = np.where(hanging, z_eff - f_throw[k], z_eff)
    xm = 0.5 * width
    iface = z0[:, None, None] + np.tan(dips)[:, None, None] * (x[None] - xm)   # [L,1,nx]
    idx = np.sum(iface < z_eff[None], axis=0)                                 # layers above
    v = v_lay[np.clip(idx, 0, n_layers)]
    v = np.where(z < z_w, v_water, v)
    return v.astype(np.float64)


def smooth(v: np.ndarray, sigma_cells: float) -> np.ndarray:
    """Starting model: Gaussian smoothing of ``v`` (std in cells, edges replicated)."""
    return gaussian_filter(v, sigma_cells, mode="nearest")


def gamma_of(v: np.ndarray) -> np.ndarray:
    """Squared slowness gamma = 1/c^2 (s^2/m^2), the model parameter of the paper."""
    return 1.0 / (v.astype(np.float64) ** 2)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

@dataclass
class Workload:
    name: str
    grid: Grid
    survey: Survey
    gamma_true: np.ndarray      # [nz, nx]
    gamma_start: np.ndarray     # [nz, nx]
    extra: dict = field(default_factory=dict)


def tiny_workload(seed: int = 0) -> Workload:
    """101x51 core at h=20 m, 10-node absorbing layer, 5 Hz, 4 sources, receivers
    in every column at depth 2; gradient + anomaly model smoothed by 10 cells."""
    g = Grid(nx=101, nz=51, npml=10, h=20.0, pml_c=3000.0)
    v = gradient_anomaly_model(g.nx, g.nz, seed=seed)
    sv = surface_survey(g.nx, 4, [5.0])
    return Workload("tiny_101x51_pml10_5Hz_4src", g, sv, gamma_of(v), gamma_of(smooth(v, 10.0)))


def marmousi_shaped_workload(seed: int = 0, n_src: int = 40, freqs=(3.0, 5.0, 7.0)) -> Workload:
    """401x141 core at h=20 m (8 km x 2.8 km), 20-node absorbing layer, layered
    faulted model smoothed by 25 cells, 40 sources, 401 receivers, 3/5/7 Hz."""
    g = Grid(nx=401, nz=141, npml=20, h=20.0, pml_c=4700.0)
    v = layered_faulted_model(g.nx, g.nz, g.h, seed=seed)
    sv = surface_survey(g.nx, n_src, list(freqs))
    return Workload(f"marmousi_shaped_401x141_pml20_{n_src}src_{len(freqs)}f", g, sv,
                    gamma_of(v), gamma_of(smooth(v, 25.0)))


def micro_workload(seed: int = 0, nx: int = 15, nz: int = 11, npml: int = 4, n_src: int = 2,
                   n_rec: int = 3, freq: float = 5.0, h: float = 20.0) -> Workload:
    """A micro grid for dense checks: 15x11 core + 4 absorbing nodes, 2 sources,
    3 receivers per source (columns spread over the surface)."""
    g = Grid(nx=nx, nz=nz, npml=npml, h=h, pml_c=3000.0)
    v = gradient_anomaly_model(nx, nz, seed=seed, sigma_cells=2.0)
    sv = surface_survey(nx, n_src, [freq])
    cols = np.linspace(0, nx - 1, n_rec).round().astype(np.int32)
    sv.rec_ix = np.tile(cols, n_src).astype(np.int32)
    sv.rec_iz = np.full(sv.rec_ix.shape, 2, dtype=np.int32)
    sv.rec_offsets = (np.arange(n_src + 1) * n_rec).astype(np.int32)
    sv.rec_w = np.ones(sv.rec_ix.shape, dtype=np.float64)
    return Workload(f"micro_{nx}x{nz}", g, sv, gamma_of(v), gamma_of(smooth(v, 3.0)))


def batching_workload(seed: int = 0) -> Workload:
    """256 sources x 2/4/6/8 Hz on the 401x141 Marmousi-shaped model
    (1024 Helmholtz blocks in one batch)."""
    return marmousi_shaped_workload(seed=seed, n_src=256, freqs=(2.0, 4.0, 6.0, 8.0))


UNEVEN_GRIDS = [(201, 71), (301, 106), (401, 141), (601, 211), (801, 281), (201, 71), (301, 106), (401, 141)]


def uneven_workloads(n_src: int = 32, freqs=(2.0, 4.0, 6.0, 8.0)) -> List[Workload]:
    """Eight independent instances of uneven grid sizes (h = 20 m, 20-node
    layer), each a seeded layered-faulted model with ``n_src`` sources."""
    out = []
    for k, (nx, nz) in enumerate(UNEVEN_GRIDS):
        g = Grid(nx=nx, nz=nz, npml=20, h=20.0, pml_c=4700.0)
        v = layered_faulted_model(nx, nz, g.h, seed=k)
        out.append(Workload(f"uneven_{k}_{nx}x{nz}", g, surface_survey(nx, n_src, list(freqs)),
                            gamma_of(v), gamma_of(smooth(v, 25.0))))
    return out


def autograd_workload(seed: int = 0) -> Workload:
    """801x281 at h = 10 m, 30-node layer, layered-faulted model, 64 sources,
    801 receivers, 6 Hz."""
    g = Grid(nx=801, nz=281, npml=30, h=10.0, pml_c=4700.0)
    v = layered_faulted_model(g.nx, g.nz, g.h, seed=seed)
    return Workload("autograd_801x281_h10_pml30_64src_6Hz", g, surface_survey(g.nx, 64, [6.0]),
                    gamma_of(v), gamma_of(smooth(v, 25.0)))


def large_workload(seed: int = 0, freqs=(4.0, 6.0, 8.0, 10.0)) -> Workload:
    """1601x561 at h = 5 m, 40-node layer, 128 sources, 1601 receivers,
    4/6/8/10 Hz (processed one frequency at a time)."""
    g = Grid(nx=1601, nz=561, npml=40, h=5.0, pml_c=4700.0)
    v = layered_faulted_model(g.nx, g.nz, g.h, seed=seed)
    return Workload("large_1601x561_h5_pml40_128src", g, surface_survey(g.nx, 128, list(freqs)),
                    gamma_of(v), gamma_of(smooth(v, 25.0)))
