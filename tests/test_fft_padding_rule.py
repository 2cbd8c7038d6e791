"""The padding rule of the FFT convolution, checked with NumPy on random
boxes: a slice's linear convolution with a kernel of half-width R,
restricted to the output box, equals the circular convolution of period P
when P >= (largest distance between an output and an input point) + R + 1
and P holds both boxes; one period shorter aliases (the bound is tight).
Input points sit at their offset from the input box's corner, kernel tap p
at p mod P, output u is read at (u - in0) mod P, one axis at a time as in
the separable 2-D transform."""
import numpy as np


def _linear(x, in0, k, R, out0, out1):
    out = np.zeros(out1 - out0)
    for o in range(out0, out1):
        for i, xi in enumerate(x):
            d = o - (in0 + i)
            if -R <= d <= R:
                out[o - out0] += xi * k[d + R]
    return out


def _circular(x, in0, k, R, out0, out1, P):
    xp = np.zeros(P)
    xp[:len(x)] = x
    kp = np.zeros(P)
    for p in range(-R, R + 1):
        kp[p % P] += k[p + R]
    y = np.fft.ifft(np.fft.fft(xp) * np.fft.fft(kp)).real
    return np.array([y[(o - in0) % P] for o in range(out0, out1)])


def _need(in0, in1, out0, out1, R):
    return max(max(out1 - 1 - in0, in1 - 1 - out0) + R + 1, in1 - in0, out1 - out0)


def test_period_from_the_rule_gives_the_linear_convolution():
    rng = np.random.default_rng(7)
    for _ in range(300):
        R = int(rng.integers(0, 12))
        in0 = int(rng.integers(0, 40))
        in1 = in0 + int(rng.integers(1, 30))
        # output boxes as the plan forms them: the input +- R, clipped to a lattice
        lo, hi = int(rng.integers(0, in0 + 1)), int(rng.integers(in1, in1 + 3 * R + 5))
        out0, out1 = max(in0 - R, lo), min(in1 + R, hi)
        if rng.random() < 0.5:   # the adjoint: input and output boxes exchanged
            in0, in1, out0, out1 = out0, out1, in0, in1
        x = rng.standard_normal(in1 - in0)
        k = rng.standard_normal(2 * R + 1)
        k = 0.5 * (k + k[::-1])   # even, like the pencil-beam kernel
        P = _need(in0, in1, out0, out1, R)
        ref = _linear(x, in0, k, R, out0, out1)
        for extra in (0, int(rng.integers(1, 9))):   # the rule's P and a larger supported size
            got = _circular(x, in0, k, R, out0, out1, P + extra)
            np.testing.assert_allclose(got, ref, atol=1e-10 * (1 + np.abs(ref).max()))


def test_one_period_shorter_aliases():
    rng = np.random.default_rng(8)
    aliased = 0
    for _ in range(200):
        R = int(rng.integers(1, 12))
        in0 = 10
        in1 = in0 + int(rng.integers(1, 30))
        out0, out1 = in0 - R, in1   # clipped on one side: the distance term binds
        P = _need(in0, in1, out0, out1, R) - 1
        if P < max(in1 - in0, out1 - out0):
            continue
        x = rng.standard_normal(in1 - in0)
        k = rng.standard_normal(2 * R + 1)
        k = 0.5 * (k + k[::-1])
        ref = _linear(x, in0, k, R, out0, out1)
        got = _circular(x, in0, k, R, out0, out1, P)
        aliased += not np.allclose(got, ref, atol=1e-8 * (1 + np.abs(ref).max()))
    assert aliased > 0
