"""Seeded workload generators (host only): the bubble array's initial fields
are the single bubble's, repeated exactly with the array's period."""
import numpy as np

import workloads as W


def test_bubble_array_repeats_the_single_bubble():
    one = W.bubble_array_2d(256, 1)
    single = dict(one)
    single.pop("array")
    a, b = W.initial_fields(one), W.initial_fields(single)
    for k in ("phi", "psi", "C"):
        assert np.array_equal(a[k], b[k]), k
    arr = W.initial_fields(W.bubble_array_2d(512, 2))
    for k in ("phi", "psi", "C"):
        f = arr[k][0]
        assert np.array_equal(f[:256, :256], a[k][0]), k
        assert np.array_equal(f[:, :256], f[:, 256:]) and np.array_equal(f[:256], f[256:]), k


def test_bubble_array_physics_is_the_bubble_rise():
    big, ref = W.bubble_array_2d(), W.bubble_rise_2d()
    for k in ("rhoR0", "rhoB0", "muR0", "muB0", "sigma0", "E0", "psi_inf", "Ds", "Db", "ra",
              "rd", "g", "R", "C0", "wall"):
        assert big[k] == ref[k], k
    assert big["nx"] == big["ny"] == 4096 and big["array"] == [16, 16, 256.0, 256.0]
