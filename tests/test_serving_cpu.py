"""Host logic of the served-stream comparison (no GPU): the first-come-
first-served completion model that the plain form is timed against."""
import numpy as np

from paper_1701_02059_gb300 import serving


def test_fifo_completion_times():
    # three jobs: the second arrives while the first is served, the third
    # after the server went idle
    services = [2.0, 1.0, 0.5]
    arrivals = [0.0, 1.0, 10.0]
    lat = serving.fifo(services, arrivals)
    assert np.allclose(lat, [2.0, 2.0, 0.5])


def test_fifo_serves_in_arrival_order_not_list_order():
    services = [1.0, 1.0]
    arrivals = [5.0, 0.0]          # the second job arrives first
    lat = serving.fifo(services, arrivals)
    assert np.allclose(lat, [1.0, 1.0])
    lat = serving.fifo([3.0, 1.0], [0.5, 0.0])
    assert np.allclose(lat, [3.5, 1.0])


def test_percentiles_summary():
    s = serving._percentiles([1.0, 2.0, 3.0, 4.0])
    assert s["p50_s"] == 2.5 and s["max_s"] == 4.0 and s["mean_s"] == 2.5
