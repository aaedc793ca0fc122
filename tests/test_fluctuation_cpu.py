"""Host arithmetic of the fluctuation measurement: dh = h - <h>_t over the
bins filled in every frame, and its RMS, against closed forms."""
import math

import numpy as np
import pytest

from paper_1701_02059_gb300.fluctuation import fluctuation


def test_standing_wave_rms_closed_form():
    """h = h0(x, y) + A sin(w t) phi(x, y) sampled at N equispaced times over
    whole periods: sum sin^2 = N / 2, so RMS = A sqrt(<phi^2>) / sqrt(2)."""
    ny, nx, T = 6, 9, 12
    y, x = np.mgrid[0:ny, 0:nx]
    h0 = 3.0 + 0.1 * x - 0.05 * y
    phi = np.cos(2 * math.pi * x / nx) * np.sin(math.pi * (y + 0.5) / ny)
    A = 0.7
    t = np.arange(T) * (2 * math.pi / T) * 2          # two whole periods
    maps = h0[None] + A * np.sin(t)[:, None, None] * phi[None]
    counts = np.full(maps.shape, 5)
    dh, rms = fluctuation(maps, counts)
    assert rms == pytest.approx(A * math.sqrt((phi ** 2).mean()) / math.sqrt(2.0), rel=1e-12)
    assert np.allclose(dh.mean(axis=0), 0.0, atol=1e-14)


def test_bins_empty_in_any_frame_are_left_out():
    rng = np.random.default_rng(0)
    maps = rng.normal(size=(5, 4, 4))
    counts = np.ones((5, 4, 4), int)
    counts[2, 1, 3] = 0                                # empty once
    maps[:, 1, 3] += 1e6                              # would dominate the RMS if kept
    dh, rms = fluctuation(maps, counts)
    assert np.isnan(dh[:, 1, 3]).all()
    keep = np.ones((4, 4), bool)
    keep[1, 3] = False
    ref = maps[:, keep] - maps[:, keep].mean(0)
    assert rms == pytest.approx(math.sqrt((ref ** 2).mean()), rel=1e-12)


def test_errors():
    with pytest.raises(ValueError):
        fluctuation(np.zeros((1, 2, 2)), np.ones((1, 2, 2)))
    with pytest.raises(ValueError):
        fluctuation(np.zeros((3, 2, 2)), np.zeros((3, 2, 2)))
