"""Discrete adjoint on the GPU: gradient of the interface mismatch after K iterations
with respect to the Robin parameters, against the oracle's adjoint and against
central differences of the GPU forward map."""
import numpy as np
import pytest

import oracle
from paper_1306_4596_gb300 import inputs

pytestmark = pytest.mark.gpu

CASES = [
    ("random_3_strips_pq", lambda: inputs.random_data(6, 12, 4, 0.05, 3, 0, True, p=[2.0, 3.0], q=[1.5, 2.5],
                                                      seed=3, nforce=1)),
    ("random_4_strips_no_bc", lambda: inputs.random_data(70, 64, 7, 0.01, 4, 0, True, p=[1.0, 4.0, 2.0], seed=4,
                                                         nforce=1, boundary_data=False)),
    ("bumps_8_strips", lambda: inputs.gaussian_bumps(64, 128, 20, 3e-3, 8, p=4.0, seed=5)),
]


def _swr():
    from paper_1306_4596_gb300 import swr
    return swr


@pytest.mark.parametrize("label,factory", CASES, ids=[c[0] for c in CASES])
def test_gradient_matches_oracle_adjoint(label, factory):
    swr = _swr()
    prob = factory()
    K = 4
    J_o, gp_o, gq_o = oracle.swr_adjoint(prob, K)
    with swr.SWR(prob) as s:
        J, gp, gq = s.gradient(K, prob.lam0)
    assert abs(J - J_o) <= 1e-11 * J_o
    scale = max(np.abs(gp_o).max(), np.abs(gq_o).max())
    assert np.abs(gp - gp_o).max() <= 1e-10 * scale, (gp, gp_o)
    assert np.abs(gq - gq_o).max() <= 1e-10 * scale, (gq, gq_o)


def test_gradient_matches_central_differences():
    swr = _swr()
    prob = inputs.gaussian_bumps(64, 128, 20, 3e-3, 8, p=[3.0, 4.0, 5.0, 4.0, 3.0, 6.0, 2.0], seed=6)
    K = 5
    with swr.SWR(prob) as s:
        J, gp, gq = s.gradient(K)
        h = 1e-5
        for j in (0, 3, 6):
            for which in ("p", "q"):
                pp, qq = prob.p.copy(), prob.q.copy()
                arr = pp if which == "p" else qq
                arr[j] += h
                s.set_robin(pp, qq)
                jp = s.gradient(K)[0]
                arr[j] -= 2 * h
                s.set_robin(pp, qq)
                jm = s.gradient(K)[0]
                fd = (jp - jm) / (2 * h)
                g = (gp if which == "p" else gq)[j]
                assert abs(g - fd) <= 1e-6 * abs(fd) + 1e-9 * J, (which, j, g, fd)
        s.set_robin(prob.p, prob.q)
        assert s.gradient(K)[0] == J


def test_set_robin_equals_fresh_handle():
    swr = _swr()
    prob = inputs.gaussian_bumps(100, 128, 15, 2e-3, 4, p=4.0, seed=8)
    newp, newq = np.array([2.0, 7.0, 3.0]), np.array([5.0, 1.5, 2.5])
    with swr.SWR(prob) as s:
        s.set_robin(newp, newq)
        s.sweep(3)
        a = (s.solution(), s.traces())
    fresh = prob.replace()
    fresh.p, fresh.q = newp, newq
    with swr.SWR(fresh) as s:
        s.sweep(3)
        b = (s.solution(), s.traces())
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_autograd_function_and_optimizer():
    import torch

    from paper_1306_4596_gb300 import adjoint
    swr = _swr()
    prob = inputs.gaussian_bumps(64, 128, 20, 3e-3, 4, p=4.0, seed=9)
    K = 4
    with swr.SWR(prob) as s:
        p = torch.tensor(prob.p, dtype=torch.float64, requires_grad=True)
        q = torch.tensor(prob.q, dtype=torch.float64, requires_grad=True)
        J = adjoint.interface_mismatch(p, q, s, K)
        J.backward()
        J0, gp, gq = oracle.swr_adjoint(prob, K)
        assert abs(J.item() - J0) <= 1e-11 * J0
        np.testing.assert_allclose(p.grad.numpy(), gp, rtol=1e-9)
        np.testing.assert_allclose(q.grad.numpy(), gq, rtol=1e-9)
        res = adjoint.optimize_robin(s, K, steps=8, lr=0.2)
        assert res["J"] < res["history"][0]["J"]


def test_gradient_rejects_unsupported():
    swr = _swr()
    with swr.SWR(inputs.small_dirichlet()) as s:
        with pytest.raises(swr.KfpError) as ei:
            s.gradient(2)
        assert ei.value.status == swr.KFP_ENOTSUP


@pytest.mark.parametrize("K", [1, 3, 11, 17])
@pytest.mark.parametrize("label,factory", CASES[1:], ids=[c[0] for c in CASES[1:]])
def test_pipelined_adjoint_equals_one_iterate_at_a_time(label, factory, K):
    """The adjoint iterates in flight together (up to 16 per launch, forward iterates
    in groups as well) give the bits of one iterate at a time, for K below, at and
    above the group size."""
    swr = _swr()
    prob = factory()
    with swr.SWR(prob, depth=1) as s:
        ref = s.gradient(K, prob.lam0)
    with swr.SWR(prob) as s:
        got = s.gradient(K, prob.lam0)
        again = s.gradient(K, prob.lam0)  # buffers reused
    for a, b, c in zip(ref, got, again):
        assert np.array_equal(np.asarray(a), np.asarray(b))
        assert np.array_equal(np.asarray(a), np.asarray(c))
