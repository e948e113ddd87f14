"""kfp_iface_norms_noalloc: the interface norms for callers that cannot allocate.

Some callers may not allocate device memory, or let a library allocate it: a
plugin inside a host application that owns every device allocation and only hands
over input and output buffers, or a latency-critical loop that cannot pay for
cudaMalloc (which can synchronise the device).  For them the library exposes the
interface-error reduction with its scratch in a fixed file-scope device array.
These tests check, through the C ABI, that two calls in a row give the norms that
kfp_swr_error reports for the same overlap values.
"""
import math

import numpy as np
import pytest

from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12  # the sums are taken in a different order than kfp_swr_error's


def _bands_and_norms(prob, iters):
    import torch
    from paper_1306_4596_gb300 import swr

    nif, ov = prob.nstrips - 1, prob.overlap
    with swr.SWR(prob) as s:
        s.sweep(iters)
        e_mis, _, j_l2, _ = swr.kfp_swr_error(s.h, 0)
        bands = torch.empty((nif, 2, prob.nt, ov + 1, prob.nx + 1), dtype=torch.float64, device="cuda")
        for j in range(nif):
            for side in range(2):
                swr.kfp_swr_bands(s.h, j, side, bands[j, side].data_ptr(), 1)
    return bands, e_mis, j_l2


@pytest.mark.parametrize("factory", [
    lambda: inputs.gaussian_bumps(300, 512, 40, 8e-4, 8, p=4.0, seed=11),
    lambda: inputs.gaussian_bumps(130, 256, 30, 1.5e-3, 4, seed=12, overlap=4, robin=False),
    # periodic x (the model problem): column nx repeats column 0 and counts once
    lambda: inputs.gaussian_bumps(119, 256, 30, 1.5e-3, 4, p=4.0, seed=13, overlap=2).replace(
        periodic_x=True, neumann_v=True),
], ids=["robin_8_strips", "dirichlet_overlap_4", "periodic_x_overlap_2"])
def test_noalloc_norms_match_kfp_swr_error(factory):
    import torch
    from paper_1306_4596_gb300 import swr

    prob = factory()
    periodic = bool(prob.periodic_x)
    ncols = prob.nx if periodic else prob.nx + 1
    nif = prob.nstrips - 1
    bands, e_mis, j_l2 = _bands_and_norms(prob, 2)
    out = torch.empty(2 + 2 * nif, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):  # the scratch array is reused from one call to the next
        out.fill_(float("nan"))
        swr.kfp_iface_norms_noalloc(bands.data_ptr(), nif, prob.nt, prob.overlap, prob.nx, prob.dt, prob.hx,
                                    out.data_ptr(), stream, periodic_x=periodic)
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        assert np.isfinite(o).all()
        assert abs(o[0] - e_mis) <= TOL * e_mis, (o[0], e_mis)
        assert abs(o[1] - j_l2) <= TOL * j_l2, (o[1], j_l2)
        per = o[2:].reshape(nif, 2)
        assert per[:, 0].max() == o[0]
        assert abs(per[:, 1].sum() - o[1]) <= TOL * o[1]
        b = bands.cpu().numpy()
        d = (b[:, 0] - b[:, 1])[..., :ncols]
        np.testing.assert_allclose(per[:, 0], np.abs(d).reshape(nif, -1).max(axis=1), rtol=0, atol=0)
        np.testing.assert_allclose(per[:, 1], prob.dt * prob.hx * (d * d).reshape(nif, -1).sum(axis=1),
                                   rtol=TOL)


def test_noalloc_rejects_more_interfaces_than_its_scratch():
    import torch
    from paper_1306_4596_gb300 import swr

    nif = swr.KFP_NOALLOC_MAX_INTERFACES + 1
    bands = torch.zeros((nif, 2, 1, 1, 2), dtype=torch.float64, device="cuda")
    out = torch.zeros(2 + 2 * nif, dtype=torch.float64, device="cuda")
    with pytest.raises(swr.KfpError) as ei:
        swr.kfp_iface_norms_noalloc(bands.data_ptr(), nif, 1, 0, 1, 0.1, 0.5, out.data_ptr(), 0)
    assert ei.value.status == swr.KFP_EINVAL
    with pytest.raises(swr.KfpError) as ei:  # a periodic grid needs two columns
        swr.kfp_iface_norms_noalloc(bands.data_ptr(), 1, 1, 0, 1, 0.1, 0.5, out.data_ptr(), 0, periodic_x=True)
    assert ei.value.status == swr.KFP_EINVAL
    assert math.isclose(out.abs().sum().item(), 0.0)
