"""Seeded test problems shared by the GPU parity tests: every input here is
generated from the oracle's density and boundary (never from the CUDA path)."""
import functools

import numpy as np
import torch

import oracle
import synth


def spec_by_name(name: str) -> synth.ModelSpec:
    """"pipipi_n30" -> the 30-knot pi pi pi model; a "_reim" suffix selects the
    Re/Im S-wave form of the same model."""
    form = "magphase"
    if name.endswith("_reim"):
        name, form = name[: -len("_reim")], "reim"
    kind, n = name.split("_n")
    return synth.model_for(kind, int(n), form)


@functools.lru_cache(maxsize=None)
def oracle_for(name: str) -> oracle.Oracle:
    return oracle.Oracle(spec_by_name(name))


@functools.lru_cache(maxsize=None)
def data_sample(name: str, n: int, seed: int = 1, f32: bool = False) -> np.ndarray:
    spec = spec_by_name(name)
    o = oracle_for(name)
    truth = synth.true_params(spec)
    dens = synth.numpy_density(lambda x: o.density(truth, x))
    dt = torch.float32 if f32 else torch.float64
    return synth.accept_reject(spec, n, dens, seed=seed, dtype=dt).numpy()


@functools.lru_cache(maxsize=None)
def uniform_sample(name: str, n: int, seed: int = 2, f32: bool = False) -> np.ndarray:
    spec = spec_by_name(name)
    o = oracle_for(name)
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    dt = torch.float32 if f32 else torch.float64
    return synth.uniform_in_plot(spec, n, ins, seed=seed, dtype=dt).numpy()


@functools.lru_cache(maxsize=None)
def grid_sample(name: str, n_side: int) -> np.ndarray:
    spec = spec_by_name(name)
    o = oracle_for(name)
    ins = synth.numpy_density(lambda x: o.inside(x).astype(np.float64))
    return synth.grid_in_plot(spec, n_side, ins).numpy()
