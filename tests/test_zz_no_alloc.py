"""adg_rhs_noalloc: the operator for callers that cannot allocate device memory.

Some callers own the whole device memory budget (a fixed arena or pool) or run a loop
where cudaMalloc's implicit synchronisation is not allowed; adg_rhs_noalloc serves them
from a built-in device scratch array instead of allocating.  These tests call it through
the C ABI and compare it with the handle-based operator adg_rhs, on two calls in a row
with different inputs (so a stale scratch would show), and with the CPU oracle's operator
(dense quadrature of Eq. 6, mass solve of Eq. 7) on the same inputs.  The file sorts last so that a
failure here cannot hide any other test.
"""
import numpy as np
import pytest

import oracle as O
from paper_2603_28710_gb300 import adg
from paper_2603_28710_gb300.inputs import random_state

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the per-step tolerance the parity tests use


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2603_28710_gb300 import build
    build.build()


def rel(a, b):
    return float(((a - b).norm() / b.norm()).item())


@pytest.mark.parametrize("dim,n_elem,p,lo,hi", [
    (2, (40, 24), 4, (-5.0, -3.0), (5.0, 3.0)),
    (3, (6, 5, 4), 3, (0.0, 0.0, 0.0), (6.0, 5.0, 4.0)),
])
def test_noalloc_matches_rhs_on_two_calls_in_a_row(dim, n_elem, p, lo, hi):
    import torch
    s = adg.Solver(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3)
    o = O.Oracle(dim=dim, n_elem=n_elem, degree=p, lo=lo, hi=hi, dt=1e-3)
    for seed in (1, 2):
        u = torch.from_numpy(random_state(s.shape, dim, seed=seed)).cuda()
        k_ref = torch.empty_like(u)
        s.rhs(u, k_ref)
        k = torch.full_like(u, float("nan"))
        adg.rhs_noalloc(dim, n_elem, p, u, k, lo=lo, hi=hi)
        torch.cuda.synchronize()
        assert torch.isfinite(k).all()
        assert rel(k, k_ref) < TOL
        ko = torch.from_numpy(o.rhs(u.cpu().numpy()))
        assert rel(k.cpu(), ko) < TOL
    s.close()


def test_noalloc_rejects_a_mesh_beyond_the_scratch_limit():
    import torch
    n_elem, p = (256, 256), 4        # needs about 63 MB of scratch, above the 32 MiB limit
    u = torch.ones((4, 256 * 256, 25), dtype=torch.float64, device="cuda")
    k = torch.empty_like(u)
    with pytest.raises(adg.AdgError) as e:
        adg.rhs_noalloc(2, n_elem, p, u, k)
    assert e.value.status == 1
    assert "limit" in str(e.value)
