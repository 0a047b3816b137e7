"""The package's Runge-Kutta tableaux (no GPU): explicit, consistent, and
satisfying the quadrature order conditions sum_i b_i c_i^(k-1) = 1/k up to the
scheme's order (4 for classic RK4, 8 for DOP853), plus the first tree
conditions beyond quadrature; unknown names are refused."""
import numpy as np
import pytest

import paper_1210_5672_gb300 as ww


@pytest.mark.parametrize("name,order,stages", [("rk4", 4, 4), ("dop853", 8, 12)])
def test_tableau_order_conditions(name, order, stages):
    a, b = ww.tableau(name)
    assert a.shape == (stages, stages) and b.shape == (stages,)
    assert np.all(np.triu(a) == 0.0)                    # explicit
    c = a.sum(axis=1)
    assert abs(b.sum() - 1.0) < 1e-14
    for k in range(1, order + 1):                       # quadrature conditions
        assert abs(b @ c ** (k - 1) - 1.0 / k) < 1e-13, k
    # tree conditions of orders 3 and 4: sum b a c = 1/6, sum b c a c = 1/8, sum b a c^2 = 1/12, sum b a a c = 1/24
    assert abs(b @ (a @ c) - 1.0 / 6.0) < 1e-13
    assert abs(b @ (c * (a @ c)) - 1.0 / 8.0) < 1e-13
    assert abs(b @ (a @ c ** 2) - 1.0 / 12.0) < 1e-13
    assert abs(b @ (a @ (a @ c)) - 1.0 / 24.0) < 1e-13


def test_dop853_is_not_of_order_nine():
    """The order-9 quadrature condition fails: the table is DOP853's 8th-order
    weights, not a higher-order pair."""
    a, b = ww.tableau("dop853")
    c = a.sum(axis=1)
    assert abs(b @ c ** 8 - 1.0 / 9.0) > 1e-8


def test_unknown_tableau_is_refused():
    with pytest.raises(ValueError):
        ww.tableau("euler")
