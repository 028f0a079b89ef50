"""The allocation-free entry point (mipwa_nll_grad_noalloc) against the
context entry point (mipwa_nll_grad), through the C ABI.

mipwa_nll_grad_noalloc is for callers that cannot allocate device memory (a
framework that owns the device heap, a serving process sized at start-up, a
plug-in whose host forbids allocation): it keeps its intermediates in one fixed
device array inside the library. Two calls in a row must both agree with the
context API within the tolerances of the parity tests (FP64: NLL 1e-12
relative, gradient 1e-8; FP32: NLL 1e-2 absolute, gradient 1e-5), which also
shows that the shared array is reset between calls. This file is collected
last so that a failure here comes after every other test has run.
"""
import numpy as np
import pytest
import torch

import synth
from tests import _problems as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1703_03284_gb300 import build
    build.build()
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")


@pytest.mark.parametrize("mode,f32", [(0, False), (1, True)], ids=["fp64", "fp32"])
def test_noalloc_matches_context_entry_point(mode, f32):
    from paper_1703_03284_gb300 import Likelihood
    from paper_1703_03284_gb300.api import nll_grad_noalloc

    name = "pipipi_n40"
    spec = P.spec_by_name(name)
    data = torch.from_numpy(P.data_sample(name, 50_000, f32=f32)).to("cuda:0")
    norm = torch.from_numpy(P.uniform_sample(name, 60_000, f32=f32)).to("cuda:0")
    lik = Likelihood(0, mode)
    lik.set_spec(spec)
    lik.set_events(data)
    lik.set_norm_sample(norm)
    for seed in (3, 4):  # two calls in a row, different parameters
        p = synth.perturbed_params(spec, seed)
        v_ref, g_ref = lik.nll_grad(p)
        v, g = nll_grad_noalloc(spec, p, data, norm, compute_mode=mode)
        gerr = np.linalg.norm(g - g_ref) / np.linalg.norm(g_ref)
        if f32:
            assert abs(v - v_ref) < 1e-2
            assert gerr < 1e-5
        else:
            assert abs(v - v_ref) <= 1e-12 * abs(v_ref)
            assert gerr < 1e-8
