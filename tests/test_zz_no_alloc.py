"""The allocation-free projector entry point (tfeti_apply_projector_noalloc).

Some callers cannot call cudaMalloc while they apply the solver's operators
(their device memory belongs to another allocator, or allocation after
start-up is forbidden).  tfeti_apply_projector_noalloc serves them by keeping its
work vectors in a static device array; this test checks through the C ABI that
it returns what tfeti_apply_projector returns, on two calls in a row (the second
call reuses the array the first one left behind).  The file name sorts last so a
run that stops at the first failure has run every other test before it.
"""
import numpy as np
import pytest

import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines only
    pytest.skip("CUDA device required", allow_module_level=True)

import paper_1205_1926_gb300 as T  # noqa: E402


@pytest.mark.parametrize("w,coarse", [(W.SMALL6_RAGGED, 0), (W.CUBE12, 0), (W.CUBE12, 2)])
def test_projector_noalloc_matches_allocating_entry_point(w, coarse):
    """Both entry points launch the same kernels in the same order on the same inputs, so
    their results are bitwise equal (the tolerance of the projector's parity tests, 1e-11, is
    checked too, as the weaker statement).  coarse = 2: the coarse solve by planes, whose
    intermediate vectors also live in the static array."""
    ctx = T.Context(w, coarse=coarse)
    m = ctx.sizes["n_mult"]
    for seed in (101, 102):
        x = torch.as_tensor(W.seeded_vector(m, seed)).cuda()
        y_ref = torch.zeros(m, dtype=torch.float64, device="cuda")
        y_static = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.apply("projector", x, y_ref)
        ctx.apply_projector_noalloc(x, y_static)
        a, b = y_static.cpu().numpy(), y_ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert np.linalg.norm(a - b) <= 1e-11 * np.linalg.norm(b)
        assert torch.equal(y_static, y_ref)


@pytest.mark.skipif(torch.cuda.device_count() < 2, reason="needs a second GPU")
def test_projector_noalloc_from_another_current_device():
    """Called while another device is current, the call still runs on the context's device and
    leaves the caller's current device as it was."""
    w = W.SMALL6_RAGGED
    ctx = T.Context(w)
    m = ctx.sizes["n_mult"]
    x = torch.as_tensor(W.seeded_vector(m, 103)).cuda(0)
    y_ref = torch.zeros(m, dtype=torch.float64, device="cuda:0")
    y_static = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda:0")
    ctx.apply("projector", x, y_ref)
    with torch.cuda.device(1):
        ctx.apply_projector_noalloc(x, y_static)
        assert torch.cuda.current_device() == 1
    assert torch.equal(y_static, y_ref)
