"""The benchmark's workload at full size, in the launch configuration the
benchmark times: the 40-knot pi pi pi model, 10^8 data and 10^8 normalisation
events stored as float32 (s12, s13), FP32-mixed NLL + gradient with computed
Breit-Wigner terms, events grouped by spline cell, one fused launch.

Inputs come from the oracle's density and boundary only: the data are a 10^7
accept-reject sample taken ten times over (repeated events are valid events),
the normalisation sample 10^8 uniform phase-space points. The oracle evaluates
the same 2 x 10^8 events in FP64. Tolerances: the stated 1e-2 absolute on
-2 ln L at 10^7 events, scaled linearly to 10^8 (1e-1), and 1e-4 norm-wise on
the gradient.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu

from paper_1703_03284_gb300 import F32, Likelihood  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


def checksum(a):
    """Order-independent checksum of an (n, 2) float32 array: sums of the bit
    patterns and of their squares (mod 2^64), equal for any permutation."""
    b = np.ascontiguousarray(a).view(np.uint32).astype(np.uint64)
    return int(b.sum(dtype=np.uint64)), int((b * b).sum(dtype=np.uint64))


def test_full_size_fp32_nll_grad_vs_oracle():
    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    data = np.tile(P.data_sample(name, 10_000_000, seed=31, f32=True), (10, 1))
    norm = synth.uniform_in_plot(
        spec, 100_000_000, synth.numpy_density(lambda x: P.oracle_for(name).inside(x).astype(np.float64)),
        seed=32, dtype=torch.float32).numpy()
    assert data.shape == norm.shape == (100_000_000, 2)
    p = synth.perturbed_params(spec, 3)
    lik = Likelihood(0, F32)
    lik.set_spec(spec)
    lik.set_events(torch.from_numpy(data))        # host buffers: copied in pieces
    lik.set_norm_sample(torch.from_numpy(norm))
    v, g = lik.nll_grad(p)
    assert abs(lik.nll(p) - v) < 1e-2  # the NLL-only kernel: same sums, own instruction schedule
    # the stored samples are permutations of the inputs
    assert checksum(lik.stored_sample("data").cpu().numpy()) == checksum(data)
    assert checksum(lik.stored_sample("norm").cpu().numpy()) == checksum(norm)
    vr, gr = P.oracle_for(name).nll_grad(p, data.astype(np.float64), norm.astype(np.float64))
    assert abs(v - vr) < 1e-1, (v, vr)
    assert np.linalg.norm(g - gr) <= 1e-4 * np.linalg.norm(gr), np.abs(g - gr).max()
