"""The seeded input generators (the stand-ins for the paper's datasets):
shapes, types and value ranges of each workload, determinism, distinct
cubes per index, exact causal prefixes where the generator promises them,
the tiny cube's planted motion, and the serving stream's arrivals."""
import numpy as np
import pytest

from paper_2506_19656_gb300 import synth


@pytest.mark.parametrize("name,T,dtype,lo,hi", [
    ("tiny", 8, np.float32, 0.0, 1.0),
    ("deepextremecubes", 3, np.float32, 0.0, 1.0),
    ("dynamicearthnet", 2, np.uint16, 0, 10000),
    ("era5", 2, np.float32, None, None),
])
def test_shape_type_and_range(name, T, dtype, lo, hi):
    c = synth.WORKLOADS[name]
    cube = synth.make_cube(name, T=T)
    assert cube.shape == (c.bands, T, c.H, c.W) and cube.dtype == dtype
    assert np.isfinite(cube.astype(np.float64)).all()
    if lo is not None:
        assert cube.min() >= lo and cube.max() <= hi
    # every band varies in space (no degenerate constant inputs)
    assert all(cube[b, 0].std() > 0 for b in range(c.bands))


@pytest.mark.parametrize("name,short,long", [("deepextremecubes", 2, 4), ("dynamicearthnet", 1, 2), ("era5", 2, 3)])
def test_causal_prefix_is_exact(name, short, long):
    assert np.array_equal(synth.make_cube(name, T=short), synth.make_cube(name, T=long)[:, :short])


def test_deterministic_and_distinct_per_cube_index():
    a = synth.make_cube("deepextremecubes", T=2)
    assert np.array_equal(a, synth.make_cube("deepextremecubes", T=2))
    assert not np.array_equal(a, synth.make_cube("deepextremecubes", cube=1, T=2))
    t0, t1 = synth.make_cube("tiny"), synth.make_cube("tiny", cube=1)
    assert not np.array_equal(t0, t1)


def test_tiny_cube_planted_motion():
    """Frame t is frame 0 moved by the cumulative step S_t, each step in
    [-4, 4]^2, so away from the borders and the noise frame t matches frame
    t-1 shifted by S_t - S_{t-1}."""
    cube, S = synth.tiny_cube(0)
    assert np.array_equal(S[0], [0, 0])
    steps = np.diff(S, axis=0)
    assert np.abs(steps).max() <= 4
    for t in range(1, cube.shape[1]):
        dx, dy = steps[t - 1]
        a = cube[:, t, 8:-8, 8:-8]
        b = cube[:, t - 1, 8 - dy:cube.shape[2] - 8 - dy, 8 - dx:cube.shape[3] - 8 - dx]
        assert np.abs(a - b).mean() < 0.01


def test_serving_stream():
    reqs = synth.serving_requests(seed=4000, n=2000, mean_interval_s=0.005)
    t = np.array([r["arrival_s"] for r in reqs])
    assert np.all(np.diff(t) > 0)
    assert np.diff(t).mean() == pytest.approx(0.005, rel=0.1)
    kinds = {k: sum(r["workload"] == k for r in reqs) for k in synth.WORKLOADS}
    assert all(400 <= n <= 600 for n in kinds.values())          # uniform over the four
    for r in reqs:
        c = synth.WORKLOADS[r["workload"]]
        assert r["qp"] in c.qps and 0 <= r["cube"] < 4
        assert r["T"] in (c.sub_T or (c.T,))
