"""ilu_inner_solve_noalloc, the allocation-free variant of the inner Schur solve.

Callers that run on a fixed device-memory budget set aside up front, or that must not
trigger the implicit synchronisation an allocation can bring, cannot let a call allocate.
This variant keeps the Krylov workspace in a fixed device array the library owns instead
of the handle's workspace. It runs the kernels of the four-launch form of ilu_inner_solve
in the same order on the same input,
so its output must equal ilu_inner_solve's bit for bit, call after call (the array keeps
the previous call's contents), and after the first call on a device neither the handle's
device memory nor torch's allocator may grow. The file is named to be collected last, so a
run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

from paper_2303_08881_gb300 import problems as P

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

@pytest.fixture(scope="module")
def ilu():
    import __graft_entry__ as g
    g.build()
    import paper_2303_08881_gb300 as m
    assert torch.cuda.is_available()
    return m




@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("k", [3, 5])
def test_noalloc_inner_solve_matches_the_handle_workspace_version(ilu, prec, k):
    pr = P.aniso2d_boxes(70, 3, seed=1)
    # the handle's own inner solve in its four-launch form: the kernels the allocation-free
    # call runs, in the same order
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision=prec, inner_iters=k, inner_launch="per_step"))
    n2 = h.sizes()["n2"]
    rng = np.random.default_rng(21)
    # a second handle on another problem between the two calls: the shared array must
    # not carry state from one call into the next
    other = ilu.ilu_setup_problem(P.convdiff3d_boxes(12, 2, seed=3), ilu.Opts(pc_precision=prec))
    n2o = other.sizes()["n2"]
    gs = [torch.from_numpy(rng.standard_normal(n2)).cuda() for _ in range(2)]
    refs = [torch.empty(n2, dtype=torch.float64, device="cuda") for _ in range(2)]
    gots = [torch.full((n2,), np.nan, dtype=torch.float64, device="cuda") for _ in range(2)]
    go = torch.from_numpy(rng.standard_normal(n2o)).cuda()
    yo = torch.empty(n2o, dtype=torch.float64, device="cuda")
    for call in range(2):
        h.inner_solve(gs[call], refs[call])
    other.inner_solve_noalloc(go, yo)   # first call on this device: looks up the array's address
    torch.cuda.synchronize()
    dev_bytes = (h.stats()["device_bytes"], other.stats()["device_bytes"])
    torch_bytes = torch.cuda.memory_allocated()
    for call in range(2):
        h.inner_solve_noalloc(gs[call], gots[call])
        torch.cuda.synchronize()
        assert torch.equal(gots[call], refs[call]), f"call {call}: max diff {(gots[call] - refs[call]).abs().max()}"
        other.inner_solve_noalloc(go, yo)
    torch.cuda.synchronize()
    assert (h.stats()["device_bytes"], other.stats()["device_bytes"]) == dev_bytes
    assert torch.cuda.memory_allocated() == torch_bytes
    assert h.stats()["device_error"] == 0
    other.close()
    h.close()


def test_noalloc_rejects_a_workspace_beyond_its_limit(ilu):
    # 512^2 grid on 16 x 16 boxes: n2 ~ 31.7k interface unknowns; FP64 with 32 inner steps
    # needs (32 + 4) * n2 * 8 B ~ 9 MB > 8 MiB
    pr = P.aniso2d_boxes(512, 16, seed=0)
    h = ilu.ilu_setup_problem(pr, ilu.Opts(pc_precision="fp64", inner_iters=32))
    n2 = h.sizes()["n2"]
    g = torch.zeros(n2, dtype=torch.float64, device="cuda")
    y = torch.zeros_like(g)
    with pytest.raises(ilu.IluError) as e:
        h.inner_solve_noalloc(g, y)
    assert e.value.status == ilu.ILU_ERR_TOO_LARGE
    h.close()
