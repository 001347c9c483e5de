"""GPU test of the allocation-free forward model (mirage_forward_noalloc).

That entry point serves callers that cannot let the library allocate device
memory (their framework owns the device-memory budget, or a cudaMalloc
would synchronise the device mid-pipeline): it takes all scratch from one
fixed array inside the library.  Here its output is compared with the
regular mirage_forward on the same inputs, twice in a row, so that the
second call also shows that nothing left in the shared array by the first
call leaks into the next result.  This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from synth import Geometry, REG_LAPLACIAN

from .helpers import device_problem, make_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_forward_twice(precision):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding

    fp32 = precision == "fp32"
    dt = torch.float32 if fp32 else torch.float64
    prec = binding.MIRAGE_FP32 if fp32 else binding.MIRAGE_FP64
    ctx = binding.Context(0, prec)
    tol = 2e-6 if fp32 else 1e-12   # the forward-model tolerance of the parity tests
    geoms = [synth.geom_ga64(), Geometry(30, 27, 0.09, 11, 13, -0.9, 0.7, -0.8, 0.9, 7, 1, REG_LAPLACIAN)]
    lenses = [[1.05, 0.65, 0.3, 0.03, -0.02, 0.04, 0.7], [0.9, 0.8, 2.0, -0.05, 0.06, 0.08, 2.9]]
    rng = np.random.default_rng(21)
    for call, (geom, lens) in enumerate(zip(geoms, lenses)):
        prob = device_problem(make_problem(geom, seed=30 + call), dt)
        L = torch.as_tensor(np.asarray(lens, dtype=np.float64), device="cuda")
        S = torch.as_tensor(rng.uniform(0, 1, (7, geom.ns)), dtype=dt, device="cuda")
        m_ref, c_ref, st_ref = ctx.forward(prob, L, S)
        m_na, c_na, st_na = binding.mirage_forward_noalloc(prec, prob, L, S)
        torch.cuda.synchronize()
        m_ref, m_na = m_ref.double().cpu().numpy(), m_na.double().cpu().numpy()
        assert int(st_na.item()) == int(st_ref.item()) == 0
        assert np.abs(m_na - m_ref).max() <= tol * np.abs(m_ref).max()
        np.testing.assert_allclose(c_na.cpu().numpy(), c_ref.cpu().numpy(), rtol=50 * tol)
    ctx.close()


def test_noalloc_rejects_oversized_problem():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding
    g = Geometry(256, 256, 0.02, 64, 64, -1.2, 1.2, -1.2, 1.2, 21, 2, REG_LAPLACIAN)  # 262144 rays
    n = g.nx * g.ny
    z = torch.zeros(n, device="cuda")
    prob = binding.Problem(g, z, torch.ones(n, device="cuda"), torch.ones(n, dtype=torch.uint8, device="cuda"),
                           torch.ones(21 * 21, device="cuda") / 441)
    with pytest.raises(binding.MirageError, match="scratch"):
        binding.mirage_forward_noalloc(binding.MIRAGE_FP32, prob, torch.tensor(synth.TRUE_LENS, device="cuda"),
                                       torch.zeros((1, g.ns), device="cuda"))
