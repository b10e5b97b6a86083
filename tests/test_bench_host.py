"""Host-side logic of bench.py that needs no GPU: the FIFO queue simulation of
the serving baseline and the CPU set of the oracle baseline."""
import os
import sys

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def test_fifo_queue():
    arrival = np.array([0.0, 0.1, 0.15, 1.0])
    service = np.array([0.2, 0.2, 0.05, 0.1])
    lat, span = bench._fifo(arrival, service)
    # 0 -> 0.2; 0.1 waits to 0.2 -> 0.4; 0.15 waits to 0.4 -> 0.45; 1.0 -> 1.1
    assert np.allclose(lat, [0.2, 0.3, 0.3, 0.1])
    assert abs(span - 1.1) < 1e-12


def test_fifo_idle_server_has_service_latency():
    arrival = np.arange(5) * 10.0
    service = np.full(5, 0.5)
    lat, span = bench._fifo(arrival, service)
    assert np.allclose(lat, 0.5) and abs(span - 40.5) < 1e-12


def test_oracle_baseline_uses_every_host_cpu():
    assert bench.HOST_CPUS_ALL == sorted(os.sched_getaffinity(0))
