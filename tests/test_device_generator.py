"""The slab-wise generator of large systems draws the same system as the
host generator (run here with torch on the CPU)."""
import numpy as np
import pytest

from synth import make_device_system, make_system


@pytest.mark.parametrize("case", [(5, 20, 60, 120, 60, 0), (7, 37, 70, 90, 45, 11)],
                         ids=lambda c: "x".join(map(str, c)))
def test_device_generator_matches_host_generator(case):
    pytest.importorskip("torch")
    s = make_system(*case)
    d = make_device_system(*case, device="cpu")
    for a, b in ((s.eps_o, d.eps_o), (s.eps_v, d.eps_v), (s.Y, d.Y), (s.x, d.x)):
        assert np.array_equal(a, b)
    assert np.abs(s.z - d.z).max() < 1e-14
    parts = list(d.cholesky_slabs(nk=7))
    assert [k0 for k0, _ in parts] == list(range(0, s.K, 7))
    L = np.concatenate([t.numpy() for _, t in parts])
    assert L.shape == s.L.shape
    # float32 vectors: a few units of float32 rounding relative to the largest entry
    assert np.abs(L - s.L).max() < 2e-6 * np.abs(s.L).max()
    assert np.array_equal(L, L.transpose(0, 2, 1))


def test_bench_generates_large_systems_in_slabs(monkeypatch):
    """bench.py takes the slab-wise generator for systems whose float64
    Cholesky array exceeds its host limit, and the host generator otherwise."""
    pytest.importorskip("torch")
    import bench
    from synth import DeviceSystem, System
    bench.set_workload("o5_v20_P60_G120_K60")
    try:
        assert isinstance(bench._system(device="cpu"), System)
        monkeypatch.setattr(bench, "HOST_L_LIMIT", 1.0)
        d = bench._system(device="cpu")
        assert isinstance(d, DeviceSystem) and d.L is None
        assert (d.o, d.v, d.P, d.G, d.K) == (5, 20, 60, 120, 60)
    finally:
        bench.set_workload(bench.DEFAULT_WORKLOAD)
