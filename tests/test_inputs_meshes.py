"""The synthetic physical meshes (inputs.annulus_mesh, inputs.square_mesh):
no triangle folds in either space, the mapped triangles tile the
computational square, and boundary vertices map onto its sides."""
import numpy as np
import pytest

from paper_2509_08109_gb300 import inputs


def _areas(P, tri):
    a, b, c = P[tri[:, 0]], P[tri[:, 1]], P[tri[:, 2]]
    return 0.5 * ((b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0]))


@pytest.mark.parametrize("make", [lambda: inputs.annulus_mesh(845, 1262), lambda: inputs.annulus_mesh(9, 13),
                                  lambda: inputs.square_mesh(27, 23, kappa_sigma=0.5)])
def test_mesh_is_valid(make):
    m = make()
    assert _areas(m.xy, m.tri).min() > 0.0
    s = _areas(m.st, m.tri)
    assert s.min() > 0.0 and abs(s.sum() - 1.0) <= 1e-12
    st_b = m.st[m.dirichlet]
    on_side = (st_b[:, 0] == 0.0) | (st_b[:, 0] == 1.0) | (st_b[:, 1] == 0.0) | (st_b[:, 1] == 1.0)
    assert on_side.all()
    st_i = m.st[~m.dirichlet]
    assert (st_i > 0.0).all() and (st_i < 1.0).all()
    assert np.all(m.f[m.dirichlet] == 0.0) and np.all(m.kappa > 0.0)
