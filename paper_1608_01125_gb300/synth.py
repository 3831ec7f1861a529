"""Seeded synthetic photon beams.

This module only draws inputs: Gaussian bunches of photons on straight lines,
shaped like the beams of the paper's Breit-Wheeler study (Sec. 3.2: two
Gaussian photon beams, head-on or crossing, MeV photons, macro-photon weights).
It holds none of the collision method's arithmetic and is imported by both the
CUDA path's callers and the CPU oracle's tests, so both see identical inputs.

Units: positions in micrometres, time in femtoseconds, energies in MeV.
Directions are unit vectors normalised here in float64; consumers take them as
given and never renormalise.

Every beam is an ``dict`` of contiguous float64 numpy arrays
``px py pz dx dy dz E w`` of equal length.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

#: speed of light in um/fs, used only to place the bunch centres so that the
#: beams meet at a chosen step.
C_UM_PER_FS = 0.299792458


@dataclasses.dataclass(frozen=True)
class BeamSpec:
    n: int
    sigma_t: tuple  # transverse (sigma_x', sigma_y') in the beam frame [um]
    sigma_l: float  # longitudinal sigma in the beam frame [um]
    divergence: float  # rms angle per transverse axis [rad]
    energy: tuple  # ("lognormal", median, sigma_ln) | ("gamma", shape, scale)
    weight: tuple = ("const", 1.0)  # ("const", w) | ("uniform", lo, hi) | ("integers", lo, hi)


@dataclasses.dataclass(frozen=True)
class Workload:
    """Two beams plus the stepping parameters of one exact run."""

    name: str
    a: BeamSpec
    b: BeamSpec
    crossing: float  # deviation from head-on [rad]; 0 = counter-propagating
    offset: float  # each centre sits this far behind the meeting point [um]
    dt: float  # [fs]
    steps: int
    kappa: float
    seed: int = 0


def _axes(crossing: float, beam: int):
    """Unit vectors (u, x', y') of a beam frame.

    Beam 0 moves along +z.  Beam 1 moves along -z rotated by ``crossing``
    about y, so the angle between the beams is pi - crossing.
    """
    if beam == 0:
        return (np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0]),
                np.array([0.0, 1.0, 0.0]))
    ca, sa = math.cos(crossing), math.sin(crossing)
    u = np.array([sa, 0.0, -ca])
    xp = np.array([ca, 0.0, sa])
    return u, xp, np.array([0.0, 1.0, 0.0])


def _draw_beam(rng: np.random.Generator, spec: BeamSpec, crossing: float,
               beam: int, offset: float) -> dict:
    n = int(spec.n)
    u, xp, yp = _axes(crossing, beam)
    # positions in the beam frame, then rotated into the lab frame
    t0 = rng.standard_normal(n) * spec.sigma_t[0]
    t1 = rng.standard_normal(n) * spec.sigma_t[1]
    lz = rng.standard_normal(n) * spec.sigma_l - offset
    # directions: normalise (tan thx, tan thy, 1) in the beam frame
    thx = rng.standard_normal(n) * spec.divergence
    thy = rng.standard_normal(n) * spec.divergence
    gx, gy = np.tan(thx), np.tan(thy)
    inv = 1.0 / np.sqrt(gx * gx + gy * gy + 1.0)
    gx, gy, gz = gx * inv, gy * inv, inv
    kind = spec.energy[0]
    if kind == "lognormal":
        E = np.exp(math.log(spec.energy[1]) + spec.energy[2] * rng.standard_normal(n))
    elif kind == "gamma":
        E = rng.gamma(spec.energy[1], spec.energy[2], n)
    elif kind == "const":
        E = np.full(n, float(spec.energy[1]))
    else:
        raise ValueError(kind)
    if spec.weight[0] == "const":
        w = np.full(n, float(spec.weight[1]))
    elif spec.weight[0] == "integers":  # macro-photons of the IP regime: lo..hi photons
        w = rng.integers(int(spec.weight[1]), int(spec.weight[2]) + 1, n).astype(np.float64)
    else:
        w = rng.uniform(spec.weight[1], spec.weight[2], n)
    out = {}
    for k, (ax, ay, az) in (("p", (t0, t1, lz)), ("d", (gx, gy, gz))):
        for c, name in enumerate("xyz"):
            out[k + name] = np.ascontiguousarray(ax * xp[c] + ay * yp[c] + az * u[c])
    out["E"] = np.ascontiguousarray(E)
    out["w"] = np.ascontiguousarray(w)
    return out


def beams(wl: Workload, seed: int | None = None) -> tuple[dict, dict]:
    """Draw beam A then beam B from ``PCG64(seed)``."""
    rng = np.random.Generator(np.random.PCG64(wl.seed if seed is None else seed))
    a = _draw_beam(rng, wl.a, wl.crossing, 0, wl.offset)
    b = _draw_beam(rng, wl.b, wl.crossing, 1, wl.offset)
    return a, b


def _spec(n, st, sl, div, energy, weight=("const", 1.0)):
    return BeamSpec(n, st, sl, div, energy, weight)


def tiny_headon(n: int = 2048, seed: int = 0) -> Workload:
    """2 x 2048 counter-propagating photons, one step of 10 fs, kappa 1e16.

    sigma_x = sigma_y = 1 um, sigma_z = 3 um, centres at -/+3 um on z,
    5 mrad divergence, log-normal energies (median 1 MeV, sigma_ln 0.5).
    """
    s = _spec(n, (1.0, 1.0), 3.0, 5e-3, ("lognormal", 1.0, 0.5))
    return Workload("headon_2x2048", s, s, 0.0, 3.0, 10.0, 1, 1e16, seed)


def headon_1m(n: int = 1 << 20, steps: int = 64, seed: int = 0) -> Workload:
    """2 x 1,048,576 photons, 64 steps of 5 fs, kappa 1e14 (FP32 + FP64 band).

    Same shape as the tiny case but sigma_z = 10 um and median energy 5 MeV.
    """
    s = _spec(n, (1.0, 1.0), 10.0, 5e-3, ("lognormal", 5.0, 0.5))
    return Workload("headon_2x1M", s, s, 0.0, 3.0, 5.0, steps, 1e14, seed)


def statistical_1e8(n: int = 100_000_000, steps: int = 32, seed: int = 0) -> Workload:
    """2 x 1e8 macro-photons, weights U[1,10], Gamma(2, 5 MeV) energies.

    sigma_r = 2 um, sigma_z = 20 um, head-on, 10 mrad, kappa 1e12, 32 steps of
    20 fs with the centres c*16*dt behind the meeting point.
    """
    s = _spec(n, (2.0, 2.0), 20.0, 10e-3, ("gamma", 2.0, 5.0), ("uniform", 1.0, 10.0))
    dt = 20.0
    return Workload("statistical_2x1e8", s, s, 0.0, C_UM_PER_FS * 16 * dt, dt, steps, 1e12, seed)


def statistical_family(i: int, n: int = 1_000_000, steps: int = 32,
                       kappa: float = 2e13) -> Workload:
    """Member ``i`` of a family of statistical workloads with varied beam
    shapes, drawn as the batching workload draws its instances: crossing
    angle U[0, pi/2], median energy log-uniform in [0.5, 50] MeV (Gamma
    spectrum of shape 2, as the statistical workload), transverse sigma
    U[0.5, 2] um.  Otherwise as the statistical workload: weights U[1, 10],
    sigma_z = 20 um, 10 mrad, steps of 20 fs with the centres c*16*dt behind
    the meeting point.  The shape is drawn from ``PCG64(2_000_003 + i)``; the
    photons from ``PCG64(3_000_017 + i)``."""
    rng = np.random.Generator(np.random.PCG64(2_000_003 + i))
    crossing = rng.uniform(0.0, math.pi / 2)
    med = math.exp(rng.uniform(math.log(0.5), math.log(50.0)))
    st = rng.uniform(0.5, 2.0)
    # the median of Gamma(2, scale) is 1.678347 scale
    s = _spec(n, (st, st), 20.0, 10e-3, ("gamma", 2.0, med / 1.6783469900166608),
              ("uniform", 1.0, 10.0))
    dt = 20.0
    return Workload(f"statistical_family_{i}", s, s, crossing, C_UM_PER_FS * 16 * dt, dt,
                    steps, kappa, 3_000_017 + i)


def crossing90_5e7(n: int = 50_000_000, steps: int = 256, seed: int = 0) -> Workload:
    """2 x 5e7 photons crossing at 90 deg, Gamma(1.5, 13.33 MeV), kappa 1e12.

    Elliptical bunches sigma_x' = 1, sigma_y' = 3, sigma_z' = 15 um in each
    beam's frame, 5 mrad, 256 steps of 2 fs, centres c*128*dt behind the
    meeting point.
    """
    s = _spec(n, (1.0, 3.0), 15.0, 5e-3, ("gamma", 1.5, 20.0 / 1.5))
    dt = 2.0
    return Workload("crossing90_2x5e7", s, s, math.pi / 2, C_UM_PER_FS * 128 * dt, dt, steps, 1e12, seed)


def batch_instance(i: int, n_min: int = 1024, n_max: int = 262144) -> Workload:
    """Instance ``i`` of the 256-instance batching workload.

    Photons per beam log-uniform in [n_min, n_max], crossing angle U[0, pi/2],
    median energy log-uniform in [0.5, 50] MeV (sigma_ln 0.5), transverse sigma
    U[0.5, 2] um, sigma_z = 3 um, 16 steps of 5 fs meeting at step 8,
    kappa 1e14, 5 mrad divergence.  The instance's shape is drawn from
    ``PCG64(i)``; its photons from ``PCG64(1_000_003 + i)``.
    """
    rng = np.random.Generator(np.random.PCG64(i))
    n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
    crossing = rng.uniform(0.0, math.pi / 2)
    med = math.exp(rng.uniform(math.log(0.5), math.log(50.0)))
    st = rng.uniform(0.5, 2.0)
    s = _spec(n, (st, st), 3.0, 5e-3, ("lognormal", med, 0.5))
    dt = 5.0
    return Workload(f"batch_{i}", s, s, crossing, C_UM_PER_FS * 8 * dt, dt, 16, 1e14,
                    1_000_003 + i)


def fixed_energy_headon(n: int, energy: float, seed: int, sigma_t: float = 1.0,
                        sigma_l: float = 3.0, offset: float = 3.0, dt: float = 10.0,
                        kappa: float = 1e16) -> Workload:
    """Zero divergence, one fixed energy: the case with a closed-form yield."""
    s = _spec(n, (sigma_t, sigma_t), sigma_l, 0.0, ("const", energy))
    return Workload("fixed_energy_headon", s, s, 0.0, offset, dt, 1, kappa, seed)


#: side of a macro-photon's cube [um] in the IP-regime workload
IP_CUBE_UM = 0.5


def ip_headon(n_mp: int = 16384, w_lo: int = 1, w_hi: int = 199, seed: int = 0) -> Workload:
    """IP regime: 2 x 16384 macro-photons of 1..199 photons each (mean 100, so
    about 1.64e6 real photons per beam), each spread over a cube of side
    IP_CUBE_UM; otherwise the 2 x 1M head-on beams (sigma = (1, 1, 10) um,
    5 mrad, log-normal energies with median 5 MeV, 64 steps of 5 fs, kappa 1e14).
    """
    s = _spec(n_mp, (1.0, 1.0), 10.0, 5e-3, ("lognormal", 5.0, 0.5), ("integers", w_lo, w_hi))
    return Workload(f"ip_headon_2x{n_mp}", s, s, 0.0, 3.0, 5.0, 64, 1e14, seed)


WORKLOADS = {
    "headon_2x2048": tiny_headon,
    "headon_2x1M": headon_1m,
    "statistical_2x1e8": statistical_1e8,
    "crossing90_2x5e7": crossing90_5e7,
}
