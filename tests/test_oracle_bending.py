"""Pins of the oracle's bending energy C_p (cost term of Eq. 1, Sec. II-F).

C_p is the thin-plate bending energy of the displacement averaged over the
image box.  Closed forms: an affine displacement has none; u_x = x^2 has
d2u/dx2 = 2 everywhere, so C_p = 4; u_y = x*y has both mixed derivatives 1,
so C_p = 2 (each counted once per order).  Cubic B-splines reproduce these
fields exactly: x = sum_j p_j beta_j(x) and x^2 = sum_j (p_j^2 - delta^2/3)
beta_j(x) with p_j = (j - 1) delta the node positions.  C_p is a quadratic
form: C_p(a c) = a^2 C_p(c) and c . grad C_p = 2 C_p; the gradient matches
central differences.
"""
import numpy as np
import pytest

from oracle.bending import bending_energy

pytestmark = pytest.mark.filterwarnings("ignore")


def node_positions(n, delta):
    nodes = (n - 1) // delta + 4
    return (np.arange(nodes) - 1.0) * delta


CASES = [((23, 17), (5, 4)), ((19, 14, 11), (4, 5, 3))]


@pytest.mark.parametrize("dims,spacing", CASES)
def test_affine_displacement_has_no_bending_energy(dims, spacing):
    nd = len(dims)
    pos = [node_positions(dims[d], spacing[d]) for d in range(nd)]
    grids = np.meshgrid(*reversed(pos), indexing="ij")[::-1]  # x, y[, z] on (.., ny, nx)
    rng = np.random.default_rng(1)
    c = np.stack([rng.normal() + sum(rng.normal() * grids[d] for d in range(nd))
                  for _ in range(nd)])
    assert abs(bending_energy(dims, spacing, c)) < 1e-18 * float(np.abs(c).max()) ** 2 + 1e-20


@pytest.mark.parametrize("dims,spacing", CASES)
def test_quadratic_and_bilinear_fields_give_closed_forms(dims, spacing):
    nd = len(dims)
    pos = [node_positions(dims[d], spacing[d]) for d in range(nd)]
    grids = np.meshgrid(*reversed(pos), indexing="ij")[::-1]
    c = np.zeros((nd,) + grids[0].shape)
    c[0] = grids[0] ** 2 - spacing[0] ** 2 / 3.0          # u_x = x^2
    assert bending_energy(dims, spacing, c) == pytest.approx(4.0, rel=1e-12)
    c = np.zeros_like(c)
    c[1] = grids[0] * grids[1]                              # u_y = x y
    assert bending_energy(dims, spacing, c) == pytest.approx(2.0, rel=1e-12)
    c[0] = grids[0] ** 2 - spacing[0] ** 2 / 3.0            # both: 4 + 2
    assert bending_energy(dims, spacing, c) == pytest.approx(6.0, rel=1e-12)


@pytest.mark.parametrize("dims,spacing", CASES)
def test_quadratic_form_scaling_euler_and_finite_differences(dims, spacing):
    nd = len(dims)
    nodes = [(dims[d] - 1) // spacing[d] + 4 for d in range(nd)]
    rng = np.random.default_rng(7)
    c = rng.normal(0.0, 1.5, (nd,) + tuple(reversed(nodes)))
    E, g = bending_energy(dims, spacing, c, grad=True)
    assert E > 0
    assert bending_energy(dims, spacing, 2.5 * c) == pytest.approx(6.25 * E, rel=1e-12)
    assert float(np.sum(c * g)) == pytest.approx(2.0 * E, rel=1e-12)
    flat = c.ravel()
    for i in rng.choice(flat.size, 12, replace=False):
        h = 1e-3
        cp = flat.copy(); cp[i] += h
        cm = flat.copy(); cm[i] -= h
        fd = (bending_energy(dims, spacing, cp.reshape(c.shape))
              - bending_energy(dims, spacing, cm.reshape(c.shape))) / (2 * h)
        # A quadratic: central differences are exact up to rounding.
        assert fd == pytest.approx(g.ravel()[i], rel=1e-7, abs=1e-10 * np.abs(g).max())
