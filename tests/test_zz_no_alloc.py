"""The allocation-free Poisson entry point gives the allocating entry point's result.

omen_poisson_static is for programs that do not let a library allocate device memory (they
hand all of it to their own allocator, or forbid allocation after start-up); it keeps its CG
work vectors in one static device array instead.  This test calls it through the C ABI twice
in a row with different charge densities (the array keeps the previous call's contents) and
compares each solution with omen_poisson's within the Poisson tolerance used by the other
tests (1e-10 of max |phi|), then checks that a grid larger than the static array is refused.
The file sorts last so that a run stopping at the first failure has run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import poisson  # noqa: E402


def _static_entry_point():
    from paper_1003_4570_gb300 import omen
    f = omen.lib().omen_poisson_static
    f.restype = C.c_int
    f.argtypes = [C.POINTER(omen.Grid), C.c_void_p, C.c_void_p, C.POINTER(omen.CGOpts),
                  C.POINTER(omen.SolveInfo), C.c_void_p]
    return f


def test_static_poisson_matches_allocating_entry_point_on_consecutive_calls():
    from paper_1003_4570_gb300 import omen
    stream = torch.cuda.current_stream().cuda_stream
    ctx = omen.omen_create(0, stream)
    solve_static = _static_entry_point()
    g = poisson.Grid(11, 11, 217, 2.1724, 2.1724, 43.448)
    gs = omen.grid_struct(g)
    opts = omen.CGOpts(1e-13, 100000)
    rng = np.random.default_rng(11)
    for _ in range(2):
        rho = torch.from_numpy(rng.normal(size=g.shape) * 1e6).cuda()
        ref = torch.zeros(g.shape, dtype=torch.float64, device="cuda")
        omen.omen_poisson(ctx, g, rho, ref, rtol=1e-13)
        phi = torch.zeros_like(ref)
        info = omen.SolveInfo()
        st = solve_static(C.byref(gs), rho.data_ptr(), phi.data_ptr(), C.byref(opts), C.byref(info), stream)
        assert st == omen.OMEN_OK and info.converged == 1
        r = ref.cpu().numpy()
        np.testing.assert_allclose(phi.cpu().numpy(), r, atol=1e-10 * np.abs(r).max(), rtol=0)
    too_big = omen.grid_struct(poisson.Grid(65, 64, 65, 10.0, 10.0, 10.0))   # 266,240 unknowns
    phi = torch.zeros(8, dtype=torch.float64, device="cuda")
    st = solve_static(C.byref(too_big), phi.data_ptr(), phi.data_ptr(), C.byref(opts), None, stream)
    assert st == omen.OMEN_EINVAL
