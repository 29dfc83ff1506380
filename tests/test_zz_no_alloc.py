"""knp_apply_preconditioner_noalloc: the allocation-free variant of knp_apply_preconditioner.

Callers that run under a CUDA stream capture, or whose host forbids allocation after
start-up, cannot let the library call cudaMalloc; this entry point keeps its work vectors in a
static device array instead. The test checks, through the C ABI, that two calls in a row give
the same result as the existing entry point, for the FP64 and the FP32 hierarchy. This file is
collected last so that a failure here leaves every other test already run.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "fp32"])
def test_noalloc_matches_apply_preconditioner(precision):
    import torch
    from paper_2403_04491_gb300 import problem_from_config
    from synth import make_config

    cfg = make_config(1)
    _, prob = problem_from_config(cfg)
    prob.amg_setup(precision=precision)
    rng = np.random.default_rng(7)
    for call in range(2):
        r = rng.standard_normal(prob.n_dof)
        z_ref = prob.apply_preconditioner(r)
        r_dev = torch.from_numpy(r).cuda()
        z_dev = torch.full_like(r_dev, float("nan"))
        prob.apply_preconditioner_noalloc(r_dev, z_dev)
        torch.cuda.synchronize()
        z = z_dev.cpu().numpy()
        # same kernels, same order: agreement to rounding of the FP64 comparison
        np.testing.assert_allclose(z, z_ref, rtol=1e-12, atol=1e-300)


def test_noalloc_rejects_a_hierarchy_beyond_the_static_array():
    import torch
    from paper_2403_04491_gb300 import KnpError, problem_from_config
    from synth import make_config

    cfg = make_config(2).with_nx(64)     # 278,683 nodes: more than the array holds in FP64
    _, prob = problem_from_config(cfg)
    prob.amg_setup(precision=0)
    r = torch.zeros(prob.n_dof, dtype=torch.float64, device="cuda")
    z = torch.zeros_like(r)
    with pytest.raises(KnpError) as ei:
        prob.apply_preconditioner_noalloc(r, z)
    assert ei.value.code == 1 and "static" in str(ei.value)
