"""GPU tests of the bending-energy penalty C_p (Eq. 1; Sec. II-F) against the
oracle's Gauss-Legendre evaluation (oracle/bending.py).

The GPU integrates with exact 1-D Gram matrices applied as FP32 stencils and
sums c . K c in FP64: C_p within 1e-5 relative, the gradient within 1e-5 of
its largest entry.  Registration with w_p > 0 reports D + w_p C_p at the
returned coefficients and lowers it; the batched driver rejects w_p > 0.
"""
import numpy as np
import pytest

import synth
from oracle.bending import bending_energy

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ("2d", synth.problem(2, (23, 17), (5, 4), (2, 2), 16)),
    ("3d", synth.problem(3, (19, 14, 11), (4, 5, 3), (2, 2, 1), 16)),
    ("ct256", synth.problem(3, (256, 256, 96), (8, 8, 8), (8, 8, 4), 64)),
]


def engine(prob, seed=3):
    import paper_1804_05061_b300 as eng
    rng = np.random.default_rng(seed)
    f = rng.random(tuple(reversed(prob.dims[:prob.ndim]))).astype(np.float32)
    m = rng.random(f.shape).astype(np.float32)
    return eng.from_problem(prob, f, m)


@pytest.mark.parametrize("name,prob", CASES)
def test_bending_energy_and_gradient_match_oracle(name, prob):
    e = engine(prob)
    c = synth.coefficients(prob, 41, 2.0)
    E_ref, g_ref = bending_energy(prob.dims[:prob.ndim], prob.ffd_spacing[:prob.ndim], c, grad=True)
    ct = torch.from_numpy(c).cuda()
    g = torch.zeros_like(ct)
    E = e.bending_energy(ct, grad_into=g, weight=1.0)
    assert abs(E - E_ref) <= 1e-5 * E_ref, (E, E_ref)
    gg = g.cpu().numpy().astype(np.float64)
    assert np.abs(gg - g_ref).max() <= 1e-5 * np.abs(g_ref).max()
    # The gradient is added to what the buffer holds, scaled by the weight.
    g2 = g.clone()
    e.bending_energy(ct, grad_into=g2, weight=0.5)
    assert torch.allclose(g2, 1.5 * g, rtol=1e-5, atol=1e-6 * float(g.abs().max()))


@pytest.mark.parametrize("name,prob", CASES[:2])
def test_quadratic_field_closed_form_on_gpu(name, prob):
    e = engine(prob)
    nd = prob.ndim
    nodes = [(prob.dims[d] - 1) // prob.ffd_spacing[d] + 4 for d in range(nd)]
    px = (np.arange(nodes[0]) - 1.0) * prob.ffd_spacing[0]
    c = np.zeros(prob.coef_shape)
    c[0] = np.broadcast_to(px ** 2 - prob.ffd_spacing[0] ** 2 / 3.0, c[0].shape)
    E = e.bending_energy(torch.from_numpy(c.astype(np.float32)).cuda())
    assert E == pytest.approx(4.0, rel=1e-4)


def test_registration_with_bending_penalty():
    import paper_1804_05061_b300 as eng
    pair = synth.make_pair("c1_2d_128")
    e = eng.from_problem(pair.prob, pair.fixed, pair.moving)
    o = e.default_opts()
    o.max_iter[0] = 20
    o.stable_window = 0
    o.penalty_weight = 0.1
    c = e.zeros()
    rep = e.register(c, 1, o)
    D = e.value(c)
    Cp = e.bending_energy(c)
    assert Cp > 0
    assert abs(rep.final_value[0] - (D + 0.1 * Cp)) <= 1e-6 * rep.final_value[0]
    assert rep.final_value[0] < e.value(e.zeros())
    # With a weight that makes the penalty as large as D at the unpenalised
    # result (C_p is ~1e-4 in voxel units here), the penalised run ends
    # smoother.
    o.penalty_weight = 0.0
    c0 = e.zeros()
    e.register(c0, 1, o)
    C0 = e.bending_energy(c0)
    o.penalty_weight = e.value(c0) / C0
    c1 = e.zeros()
    e.register(c1, 1, o)
    assert e.bending_energy(c1) < C0


def test_batched_driver_rejects_a_penalty():
    import paper_1804_05061_b300 as eng
    specs = synth.batch_specs(2, seed=77, edges=(24, 40))
    b = eng.Batch([eng.from_problem(s.prob, s.fixed, s.moving, storage="f32") for s in specs])
    o = eng.SRWCR.default_opts()
    o.penalty_weight = 0.1
    with pytest.raises(eng.SrwcrError, match="EINVAL"):
        b.register(o)
