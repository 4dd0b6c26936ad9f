"""Pins for the paper-literal temperature path (Sec. 3.3.3): the temperature is
recovered from the reconstructed green channel through the colour-temperature
table.  The green channel grows with temperature over 800-2000 K (the paper's
reason for choosing it), the inverse undoes the table's interpolant exactly,
reproduces the table's own nodes, and clamps outside the range."""
import numpy as np
import pytest

T_MIN, T_MAX, M = 800.0, 2000.0, 1024


@pytest.fixture(scope="module")
def lut(orc):
    return orc.lut_build(T_MIN, T_MAX, M)


def test_green_grows_with_temperature(orc, lut):
    assert np.all(np.diff(lut[:, 1]) > 0)
    # and so does the Planck-integrated green response itself, off the table nodes
    t = np.linspace(T_MIN, T_MAX, 97)
    g = np.array([orc.temp_rgb(x)[1] for x in t])
    assert np.all(np.diff(g) > 0)


def test_inverse_of_the_table_interpolant(orc, lut):
    rng = np.random.default_rng(3)
    t = rng.uniform(T_MIN, T_MAX, size=400)
    # the table's piecewise-linear green at t, written from the table rows
    u = (t - T_MIN) / (T_MAX - T_MIN) * (M - 1)
    i = np.minimum(np.floor(u).astype(int), M - 2)
    f = u - i
    g = lut[i, 1] + f * (lut[i + 1, 1] - lut[i, 1])
    back = orc.green_to_temp(g, lut, T_MIN, T_MAX)
    np.testing.assert_allclose(back, t, rtol=0, atol=1e-7)


def test_table_nodes_and_clamping(orc, lut):
    nodes = T_MIN + np.arange(M) * (T_MAX - T_MIN) / (M - 1)
    back = orc.green_to_temp(lut[:, 1], lut, T_MIN, T_MAX)
    np.testing.assert_allclose(back, nodes, rtol=0, atol=1e-9)
    assert orc.green_to_temp(np.array([0.0, -1.0, lut[0, 1] * 0.5]), lut, T_MIN, T_MAX).tolist() == [T_MIN] * 3
    assert orc.green_to_temp(np.array([lut[-1, 1] * 2.0, 1e30]), lut, T_MIN, T_MAX).tolist() == [T_MAX] * 2


def test_green_of_planck_at_the_table_range(orc, lut):
    """The table's green at 2000 K is the normalisation (1) and its green at
    800 K is far smaller: a dim background maps to the bottom of the range."""
    assert lut[-1, 1] == pytest.approx(1.0, rel=1e-12)
    assert lut[0, 1] < 1e-6
