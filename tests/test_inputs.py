"""The seeded input recipe (paper_2303_02543_gb300/inputs.py) against its
published definitions and stated distributions: the generator is shared by
the CUDA path and the oracle, so these checks pin what both sides are fed."""
import math

import numpy as np

from paper_2303_02543_gb300 import inputs

MASK = (1 << 64) - 1


def splitmix64_reference(state, n):
    """splitmix64 written out on Python integers from its published
    definition (Steele, Lea and Flood 2014): add the golden gamma to the
    state, then the two xor-shift-multiply rounds and a final xor-shift."""
    out = []
    for _ in range(n):
        state = (state + 0x9E3779B97F4A7C15) & MASK
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_its_definition_and_published_outputs():
    # from state 0 the generator's first outputs are widely published
    ref = splitmix64_reference(0, 3)
    assert ref == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    ctr = np.arange(1, 4, dtype=np.uint64) * inputs._GAMMA
    assert [int(v) for v in inputs._mix(ctr)] == ref
    # a keyed stream is the same recurrence started from the key
    key = int(inputs._key(2305, 7))
    assert [int(v) for v in inputs.u64_stream(2305, 7, 5)] == splitmix64_reference(key, 5)
    assert [int(v) for v in inputs.u64_stream(2305, 7, 2, start=3)] == splitmix64_reference(key, 5)[3:]


def test_streams_are_deterministic_and_distinct_per_array():
    a = inputs.u64_stream(11, 1, 1000)
    assert np.array_equal(a, inputs.u64_stream(11, 1, 1000))
    for other in (inputs.u64_stream(11, 2, 1000), inputs.u64_stream(12, 1, 1000)):
        assert np.count_nonzero(a == other) == 0


def test_uniform_is_top_53_bits_and_uniform():
    u = inputs.uniform(5, 3, 200000)
    raw = inputs.u64_stream(5, 3, 200000)
    assert np.array_equal(u, (raw >> np.uint64(11)).astype(np.float64) * 2.0 ** -53)
    assert u.min() >= 0.0 and u.max() < 1.0
    # mean 1/2 and variance 1/12 within five standard errors
    n = u.size
    assert abs(u.mean() - 0.5) < 5 * math.sqrt(1 / 12 / n)
    assert abs(u.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / n)


def test_normal_has_unit_moments():
    z = inputs.normal(6, 4, 400000)
    n = z.size
    assert abs(z.mean()) < 5 / math.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * math.sqrt(2 / n)
    # tails of a standard normal: P(|z| > 3) = 0.0027
    assert abs(np.mean(np.abs(z) > 3.0) - 0.0027) < 0.0006


def test_problem_shapes_and_face_sizes():
    for dims in ((7, 5), (7, 5, 3)):
        p = inputs.make_problem(dims, dims, 9, boundary="uniform", source="normal", x0="uniform")
        assert p.source.shape == tuple(reversed(dims)) and p.x0.shape == p.source.shape
        assert [f.size for f in p.faces] == list(inputs.face_shapes(dims))
        n = list(dims) + [1] * (3 - len(dims))
        assert list(inputs.face_shapes(dims)) == [n[1] * n[2], n[1] * n[2], n[0] * n[2], n[0] * n[2],
                                                  n[0] * n[1], n[0] * n[1]][:2 * len(dims)]


def test_batched_recipe_sides_are_log_uniform_within_bounds():
    sides = inputs.log_uniform_sides(2307, 100, 20000, 64, 2048)
    assert sides.min() >= 64 and sides.max() <= 2048
    # log(side) uniform: its median is the geometric mean of the bounds
    assert abs(np.median(np.log(sides)) - 0.5 * (math.log(64) + math.log(2048))) < 0.05
    probs = inputs.batched_2d(count=16, size_scale=0.25)
    for q in probs:
        assert all(1 <= b <= d for b, d in zip(q.block, q.dims))


def test_serving_arrivals_are_poisson_at_the_rate():
    stream = inputs.serving_stream(rate=50.0, window_s=200.0, lo2=8, hi2=16, lo3=4, hi3=8)
    t = np.array([a.t for a in stream])
    assert np.all(np.diff(t) > 0) and t[-1] <= 200.0
    gaps = np.diff(np.concatenate([[0.0], t]))
    # exponential gaps: mean 1/rate, standard deviation equal to the mean
    n = gaps.size
    assert abs(gaps.mean() - 1 / 50.0) < 5 * (1 / 50.0) / math.sqrt(n)
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.05
    kinds = np.array([a.problem.ndim for a in stream])
    assert abs(np.mean(kinds == 3) - 0.5) < 5 * math.sqrt(0.25 / n)
