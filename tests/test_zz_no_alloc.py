"""GPU test of the allocation-free forward model (mirage_forward_noalloc).

That entry point serves callers that cannot let the library allocate device
memory (their framework owns the device-memory budget, or a cudaMalloc
would synchronise the device mid-pipeline): it takes all scratch from one
fixed array inside the library.  Its output is compared with the regular
mirage_forward on the same inputs, twice in a row, so that the second call
also shows that nothing left in the shared array by the first call leaks
into the next result; and directly with the CPU oracle's B L s and chi^2.
One case has more sources than the entry point's 32 CTAs, so a CTA loops
over several sources and reuses its image slab in the fixed array.  This
file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import synth
from oracle.solve import forward_chi2
from synth import Geometry, REG_LAPLACIAN

from .helpers import device_problem, make_problem

pytestmark = pytest.mark.gpu

# (geometry, lens, number of sources): the 64x64 workload with 7 sources,
# a ragged 30x27 image with 7, and the 64x64 workload with 41 sources (more
# than the 32 CTAs of the allocation-free launch)
CASES = [
    (synth.geom_ga64(), [1.05, 0.65, 0.3, 0.03, -0.02, 0.04, 0.7], 7),
    (Geometry(30, 27, 0.09, 11, 13, -0.9, 0.7, -0.8, 0.9, 7, 1, REG_LAPLACIAN),
     [0.9, 0.8, 2.0, -0.05, 0.06, 0.08, 2.9], 7),
    (synth.geom_ga64(), [0.95, 0.75, 1.2, -0.04, 0.05, 0.02, 0.4], 41),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_noalloc_matches_forward_and_oracle(precision):
    import __graft_entry__
    __graft_entry__.build()
    from paper_1101_5803_gb300 import binding

    fp32 = precision == "fp32"
    dt = torch.float32 if fp32 else torch.float64
    prec = binding.MIRAGE_FP32 if fp32 else binding.MIRAGE_FP64
    ctx = binding.Context(0, prec)
    tol = 2e-6 if fp32 else 1e-12   # the forward-model tolerance of the parity tests
    rng = np.random.default_rng(21)
    for call, (geom, lens, n_src) in enumerate(CASES):
        hprob = make_problem(geom, seed=30 + call)
        prob = device_problem(hprob, dt)
        L = torch.as_tensor(np.asarray(lens, dtype=np.float64), device="cuda")
        S_h = rng.uniform(0, 1, (n_src, geom.ns))
        if fp32:
            S_h = S_h.astype(np.float32).astype(np.float64)
        S = torch.as_tensor(S_h, dtype=dt, device="cuda")
        m_ref, c_ref, st_ref = ctx.forward(prob, L, S)
        # two allocation-free calls in a row on the same inputs
        outs = [binding.mirage_forward_noalloc(prec, prob, L, S) for _ in range(2)]
        torch.cuda.synchronize()
        m_ref = m_ref.double().cpu().numpy()
        m_o, c_o = forward_chi2(hprob, lens, S_h)
        scale = np.abs(m_o).max()
        for m_na, c_na, st_na in outs:
            m_na = m_na.double().cpu().numpy()
            c_na = c_na.cpu().numpy()
            assert int(st_na.item()) == int(st_ref.item()) == 0
            assert np.abs(m_na - m_ref).max() <= tol * np.abs(m_ref).max()
            np.testing.assert_allclose(c_na, c_ref.cpu().numpy(), rtol=50 * tol)
            # against the oracle's explicit B L s and its chi^2, every source
            assert np.abs(m_na - m_o).max() <= tol * scale
            np.testing.assert_allclose(c_na, c_o, rtol=50 * tol)
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
