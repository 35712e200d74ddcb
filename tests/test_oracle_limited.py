"""The limited-view workload generator and its data recipe (no inverse
crime): sensors sit in rows/columns just inside the absorbing layer, x_true
is the block mean of the fine phantom, and data simulated by the FP64 oracle
on the twice-finer grid (half the time step, every second sample) agree with
the coarse model's data to discretisation accuracy but not exactly."""
import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("sides", [1, 2])
def test_limited_view_layout(sides):
    w = synth.workload("limited", n=64, sides=sides)
    ex = w.extra
    assert w.ns == 80 and w.shape == (64, 64)
    d = (ex["layer"] + 1) * w.h
    on_top = np.isclose(w.sensors[:, 1], d)
    on_left = np.isclose(w.sensors[:, 0], d)
    assert on_top.sum() == (80 if sides == 1 else 40)
    assert (on_top | on_left).all()
    assert ex["x_fine"].shape == (128, 128)
    np.testing.assert_allclose(w.x_true, ex["x_fine"].reshape(64, 2, 64, 2).mean(axis=(1, 3)))
    assert ex["nt_fine"] == 2 * (w.nt - 1) + 1
    np.testing.assert_allclose(ex["dt_fine"] * 2, w.dt)


def test_fine_grid_data_close_to_coarse_model():
    w = synth.workload("limited", n=48)
    ex = w.extra
    smax = oracle.sponge_sigma_max(1500.0, ex["layer"], w.h)
    fine = oracle.Wave((96, 96), ex["h_fine"], ex["dt_fine"], ex["nt_fine"], w.order, 1500.0, w.sensors,
                       sigma=oracle.sponge_sigma((96, 96), 2 * ex["layer"], smax))
    coarse = oracle.Wave(w.shape, w.h, w.dt, w.nt, w.order, 1500.0, w.sensors,
                         sigma=oracle.sponge_sigma(w.shape, ex["layer"], smax))
    y_f = fine.forward(ex["x_fine"])[:, ::2]
    y_c = coarse.forward(w.x_true)
    r = np.linalg.norm(y_f - y_c) / np.linalg.norm(y_c)
    assert 1e-4 < r < 0.25
