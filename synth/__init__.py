"""Seeded synthetic inputs for the MIPWA likelihood: decay models, true parameter
points, and generic samplers.

This module holds no amplitude, kinematics or likelihood arithmetic. Where a
sample has to follow the Dalitz-plot PDF (accept-reject, Sec. 4 of
arXiv:1703.03284: toy samples generated from the Dalitz-plot PDF) or be
restricted to the Dalitz plot, the caller passes the density or the
inside-indicator as a function; the sampler only draws random numbers, builds a
piecewise-constant envelope from the values it is given and applies the
accept step. Tests pass the oracle's functions; the benchmark passes the
library's own.

Workload recipe (the paper's LHCb sample is not available; these stand in for it):
  * D+ -> pi- pi+ pi+ with rho(770) (P-wave) and f2(1270) (D-wave), or
    D+ -> K- pi+ pi+ with K*(892) (P-wave) and K2*(1430) (D-wave);
  * Blatt-Weisskopf radii 1.5/GeV (resonance) and 5.0/GeV (D meson);
  * S-wave knots uniform in m^2(h1 h2) over the stated range; true magnitudes
    1 + 0.5 sin(k) and phases rising linearly from 0 to 3 rad (k = 0..N-1);
  * true BW coefficients c_P = 0.2 (held fixed as the reference) and
    c_D = 0.3 exp(1.0 i);
  * data drawn by accept-reject from |A|^2; normalisation samples uniform over
    the Dalitz plot, or the in-boundary centres of an evenly spaced grid.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, Sequence

import numpy as np
import torch

M_D = 1.86966
M_PI = 0.13957
M_K = 0.493677


@dataclasses.dataclass(frozen=True)
class ModelSpec:
    """D -> h1 h2 h3 with m3 = m2 (the two identical particles)."""

    name: str
    mD: float
    m1: float
    m2: float
    resonances: tuple  # ((mass, width, spin), ...)
    knots: tuple       # strictly increasing s_k in GeV^2
    r_res: float = 1.5
    r_D: float = 5.0
    fixed: tuple = (0, 1)  # parameter indices held fixed in fits (Re c_0, Im c_0)
    # S-wave knot values: "magphase" = (a_k, phi_k), "reim" = (Re, Im) of a_k e^{i phi_k}
    swave_form: str = "magphase"

    @property
    def n_res(self) -> int:
        return len(self.resonances)

    @property
    def n_knots(self) -> int:
        return len(self.knots)

    @property
    def n_params(self) -> int:
        return 2 * self.n_res + 2 * self.n_knots

    @property
    def s_lo(self) -> float:
        """Lower edge of the bounding square, (m1 + m2)^2."""
        return (self.m1 + self.m2) ** 2

    @property
    def s_hi(self) -> float:
        """Upper edge of the bounding square, (mD - m3)^2."""
        return (self.mD - self.m2) ** 2


def uniform_knots(lo: float, hi: float, n: int) -> tuple:
    return tuple(float(x) for x in np.linspace(lo, hi, n))


def pipipi(n_knots: int) -> ModelSpec:
    """D+ -> pi- pi+ pi+, rho(770) P-wave + f2(1270) D-wave + MIPWA S-wave."""
    return ModelSpec(
        name=f"pipipi_n{n_knots}", mD=M_D, m1=M_PI, m2=M_PI,
        resonances=((0.77526, 0.1491, 1), (1.2755, 0.1867, 2)),
        knots=uniform_knots(0.078, 2.987, n_knots))


def kpipi(n_knots: int) -> ModelSpec:
    """D+ -> K- pi+ pi+, K*(892) P-wave + K2*(1430) D-wave + MIPWA K pi S-wave."""
    lo = (M_K + M_PI) ** 2
    hi = (M_D - M_PI) ** 2
    return ModelSpec(
        name=f"kpipi_n{n_knots}", mD=M_D, m1=M_K, m2=M_PI,
        resonances=((0.89555, 0.0473, 1), (1.4324, 0.109, 2)),
        knots=uniform_knots(lo, hi, n_knots))


def kkk(n_knots: int = 40) -> ModelSpec:
    """D+ -> K- K+ K+ (Sec. 4): phi(1020) P-wave + MIPWA K+K- S-wave with knots
    over the whole m^2(K+K-) range. The phi mass and width are not in the paper;
    these are the world-average values (1019.461 MeV, 4.249 MeV)."""
    lo = (2 * M_K) ** 2
    hi = (M_D - M_K) ** 2
    return ModelSpec(name=f"kkk_n{n_knots}", mD=M_D, m1=M_K, m2=M_K,
                     resonances=((1.019461, 0.004249, 1),),
                     knots=uniform_knots(lo, hi, n_knots))


def pipipi_isobar() -> ModelSpec:
    """Isobar baseline of the pi pi S-wave (the model a MIPWA replaces, Sec. 1-2):
    rho(770) P, f2(1270) D and two scalar Breit-Wigner terms, f0(980) and
    f0(1370); the spline is kept with two knots whose values are held at zero
    (A0 = 0). The paper gives no f0 parameters: 0.990 GeV / 0.055 GeV and
    1.350 GeV / 0.350 GeV are used."""
    lo, hi = 0.078, 2.987
    res = ((0.77526, 0.1491, 1), (1.2755, 0.1867, 2), (0.990, 0.055, 0), (1.350, 0.350, 0))
    return ModelSpec(name="pipipi_isobar", mD=M_D, m1=M_PI, m2=M_PI, resonances=res,
                     knots=(lo, hi), fixed=(0, 1, 8, 9, 10, 11))


def as_reim(spec: ModelSpec) -> ModelSpec:
    """The same decay model with the S-wave knot values taken as real and
    imaginary parts (the complex-plane spline of Sec. 2 read literally)."""
    return dataclasses.replace(spec, name=spec.name + "_reim", swave_form="reim")


def true_params(spec: ModelSpec) -> np.ndarray:
    """[Re c_0, Im c_0, ..., a_0..a_{N-1}, phi_0..phi_{N-1}]; for the Re/Im form
    the knot block is [a_k cos phi_k..., a_k sin phi_k...] (the same complex
    knot values)."""
    if spec.name.startswith("kkk"):
        # c_phi = 0.06: the phi makes ~10 % of the rate, the S-wave the rest (Sec. 4)
        c = [0.06 + 0.0j]
    elif spec.name == "pipipi_isobar":
        c = [0.2 + 0.0j, 0.3 * complex(math.cos(1.0), math.sin(1.0)),
             0.1 * complex(math.cos(0.5), math.sin(0.5)),
             0.1 * complex(math.cos(-0.5), math.sin(-0.5))]
        return np.array([v for z in c for v in (z.real, z.imag)] + [0.0] * (2 * spec.n_knots))
    else:
        c = [0.2 + 0.0j, 0.3 * complex(math.cos(1.0), math.sin(1.0))]
    c = (c + [0.1 + 0.0j] * spec.n_res)[: spec.n_res]
    n = spec.n_knots
    a = [1.0 + 0.5 * math.sin(k) for k in range(n)]
    phi = [3.0 * k / (n - 1) for k in range(n)]
    out = []
    for z in c:
        out += [z.real, z.imag]
    if spec.swave_form == "reim":
        a, phi = ([ak * math.cos(pk) for ak, pk in zip(a, phi)],
                  [ak * math.sin(pk) for ak, pk in zip(a, phi)])
    return np.array(out + a + phi, dtype=np.float64)


def perturbed_params(spec: ModelSpec, seed: int, scale: float = 0.05) -> np.ndarray:
    """True parameters moved off the truth, so that the gradient is not ~0."""
    rng = np.random.default_rng(seed)
    p = true_params(spec)
    return p + scale * rng.standard_normal(p.shape)


# ------------------------------------------------------------------ samplers
Density = Callable[[torch.Tensor], torch.Tensor]


def _gen(seed: int, device) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def _round(x: torch.Tensor, dtype) -> torch.Tensor:
    """Round candidates to the storage dtype before any density is evaluated, so
    accepted events are exactly representable in it."""
    if dtype == torch.float32:
        return x.to(torch.float32).to(torch.float64)
    return x


def uniform_in_plot(spec: ModelSpec, n: int, inside: Density, seed: int,
                    device="cpu", dtype=torch.float64, chunk: int = 1 << 22) -> torch.Tensor:
    """n points uniform over the Dalitz plot: uniform in the bounding square,
    kept where ``inside`` (a 0/1 indicator) is non-zero."""
    g = _gen(seed, device)
    lo, hi = spec.s_lo, spec.s_hi
    out, have = [], 0
    while have < n:
        x = lo + (hi - lo) * torch.rand((chunk, 2), generator=g, device=device,
                                        dtype=torch.float64)
        x = _round(x, dtype)
        keep = inside(x) > 0
        x = x[keep]
        out.append(x)
        have += x.shape[0]
    return torch.cat(out)[:n].to(dtype)


def grid_centres(spec: ModelSpec, n_side: int, device="cpu") -> torch.Tensor:
    """Centres of an n_side x n_side lattice of equal cells over the bounding
    square (the caller keeps the in-boundary ones)."""
    lo, hi = spec.s_lo, spec.s_hi
    step = (hi - lo) / n_side
    c = lo + step * (torch.arange(n_side, dtype=torch.float64, device=device) + 0.5)
    a, b = torch.meshgrid(c, c, indexing="ij")
    return torch.stack([a.reshape(-1), b.reshape(-1)], dim=1)


def grid_in_plot(spec: ModelSpec, n_side: int, inside: Density, device="cpu") -> torch.Tensor:
    pts = grid_centres(spec, n_side, device)
    return pts[inside(pts) > 0]


def spacing_grid_in_plot(spec: ModelSpec, spacing: float, inside: Density,
                         device="cpu") -> torch.Tensor:
    """Evenly spaced grid with the given spacing in GeV^2 (normalisation grids of
    Sec. 4, Fig. 2: 0.01, 0.004, 0.001)."""
    n_side = int(math.ceil((spec.s_hi - spec.s_lo) / spacing))
    return grid_in_plot(spec, n_side, inside, device)


class EnvelopeError(RuntimeError):
    pass


def accept_reject(spec: ModelSpec, n: int, density: Density, seed: int, device="cpu",
                  dtype=torch.float64, cells: int = 64, scan: int = 8,
                  safety: float = 1.5, chunk: int = 1 << 21) -> torch.Tensor:
    """n events distributed as ``density`` (zero outside the Dalitz plot).

    The envelope is piecewise constant on a cells x cells lattice over the
    bounding square: safety x the largest density value seen on a scan x scan
    sub-lattice of each cell (cell edges included). Candidates are drawn cell by
    cell with probability proportional to the envelope, then uniformly inside
    the cell, and accepted when u * envelope < density. A candidate whose density
    exceeds its envelope raises EnvelopeError.
    """
    g = _gen(seed, device)
    lo, hi = spec.s_lo, spec.s_hi
    w = (hi - lo) / cells
    # scan lattice: (cells*scan + 1)^2 points, cell (i, j) covers sub-points
    # [i*scan, (i+1)*scan] x [j*scan, (j+1)*scan]
    m = cells * scan + 1
    t = lo + (hi - lo) * torch.arange(m, dtype=torch.float64, device=device) / (m - 1)
    a, b = torch.meshgrid(t, t, indexing="ij")
    f = density(torch.stack([a.reshape(-1), b.reshape(-1)], 1)).reshape(m, m)
    fmax = torch.zeros(cells, cells, dtype=torch.float64, device=device)
    for di in range(scan + 1):
        for dj in range(scan + 1):
            sub = f[di: di + cells * scan: scan, dj: dj + cells * scan: scan]
            fmax = torch.maximum(fmax, sub)
    # cells touching the plot but whose scan points all fell outside still get an
    # envelope from their neighbours
    pad = torch.nn.functional.pad(fmax[None, None], (1, 1, 1, 1))
    neigh = torch.nn.functional.max_pool2d(pad, 3, stride=1)[0, 0]
    env = safety * torch.maximum(fmax, neigh).reshape(-1)
    prob = env / env.sum()
    out, have = [], 0
    while have < n:
        cell = torch.multinomial(prob, chunk, replacement=True, generator=g)
        u = torch.rand((chunk, 3), generator=g, device=device, dtype=torch.float64)
        ci = torch.div(cell, cells, rounding_mode="floor").to(torch.float64)
        cj = (cell % cells).to(torch.float64)
        x = torch.stack([lo + w * (ci + u[:, 0]), lo + w * (cj + u[:, 1])], 1)
        x = _round(x, dtype)
        fx = density(x)
        e = env[cell]
        if bool((fx > e).any()):
            raise EnvelopeError("density exceeds the accept-reject envelope")
        keep = u[:, 2] * e < fx
        x = x[keep]
        out.append(x)
        have += x.shape[0]
    return torch.cat(out)[:n].to(dtype)


def toy_sizes(n_toys: int, seed: int, lo_exp: float = 4.0, hi_exp: float = 6.0) -> np.ndarray:
    """Toy event counts: Poisson around means log-uniform in [10^lo, 10^hi]."""
    rng = np.random.default_rng(seed)
    mu = 10.0 ** rng.uniform(lo_exp, hi_exp, size=n_toys)
    return rng.poisson(mu).astype(np.int64)


def numpy_density(fn: Callable[[np.ndarray], np.ndarray]) -> Density:
    """Adapt a numpy (n,2)->(n,) function (such as the oracle's) to a Density."""
    def f(x: torch.Tensor) -> torch.Tensor:
        return torch.from_numpy(np.asarray(fn(x.detach().cpu().numpy()), dtype=np.float64)).to(x.device)
    return f


CONFIGS = {
    # small case the oracle finishes in seconds: 10^4 events, 100x100 grid
    "pipipi_n10_1e4_grid100": dict(model=("pipipi", 10), n_data=10_000, norm=("grid", 100),
                                   dtype="f64", seed_data=1, seed_norm=2),
    # full fit: 10^6 + 10^6 float64 events, 30 knots
    "pipipi_n30_1e6": dict(model=("pipipi", 30), n_data=1_000_000, norm=("uniform", 1_000_000),
                           dtype="f64", seed_data=1, seed_norm=2),
    # precision form: 10^8 + 10^8 float32 events, 40 knots
    "pipipi_n40_1e8_f32": dict(model=("pipipi", 40), n_data=100_000_000,
                               norm=("uniform", 100_000_000), dtype="f32",
                               seed_data=1, seed_norm=2),
    # differentiation: 10^7 events, 40 knots, pi pi pi and K pi pi
    "pipipi_n40_1e7": dict(model=("pipipi", 40), n_data=10_000_000, norm=("uniform", 10_000_000),
                           dtype="f64", seed_data=1, seed_norm=2),
    "kpipi_n40_1e7": dict(model=("kpipi", 40), n_data=10_000_000, norm=("uniform", 10_000_000),
                          dtype="f64", seed_data=1, seed_norm=2),
}


def model_for(kind: str, n_knots: int, swave_form: str = "magphase") -> ModelSpec:
    spec = {"pipipi": pipipi, "kpipi": kpipi, "kkk": kkk}[kind](n_knots)
    return as_reim(spec) if swave_form == "reim" else spec
