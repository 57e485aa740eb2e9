"""The float64 pivot reciprocal of the factorisation kernels against CUDA's
correctly rounded quotient.

The kernels form 1/d from the PTX estimate rcp.approx.ftz.f64 refined by a
cubic Newton-Raphson step.  The stated bound is checked here over normal d
spanning the exponent range: every result within one ulp of 1/d.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1402_5056_gb300 import binding as b  # noqa: E402


def test_reciprocals_within_their_bounds():
    rng = np.random.default_rng(1402)
    d = np.concatenate([
        10.0 ** rng.uniform(-300, 300, 200000),             # the exponent range
        rng.uniform(0.5, 2.0, 200000),                      # around 1 (pivots of Gram matrices)
        2.0 ** np.arange(-1020, 1021, dtype=np.float64),    # powers of two: exact reciprocals
        np.nextafter(2.0 ** np.arange(-60, 61, dtype=np.float64), np.inf),
        np.nextafter(2.0 ** np.arange(-60, 61, dtype=np.float64), 0.0),
    ])
    dd = torch.from_numpy(d).cuda()
    quot = (1.0 / dd).cpu().numpy()                         # CUDA's IEEE division
    pr = torch.empty_like(dd)
    ctx = b.h2_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        b.h2_check_reciprocal(ctx, dd.data_ptr(), len(d), pr.data_ptr())
        b.h2_ctx_synchronize(ctx)
    finally:
        b.h2_ctx_destroy(ctx)
    pr = pr.cpu().numpy()
    np.testing.assert_array_equal(quot, 1.0 / d)           # host and device agree on 1/d
    ulp = np.spacing(np.abs(quot))
    assert np.all(np.abs(pr - quot) <= ulp), float(np.max(np.abs(pr - quot) / ulp))
    # most of the cubic form's results are the correctly rounded quotient
    assert np.mean(pr == quot) > 0.9
