"""The arithmetic identities the bootstrapped circuit's scalar chain rests on,
in plain FP64 (CPU):

- the coupled Goldschmidt pair (g, h) carried as one complex constant
  z = g + i h/4: 2 Im(z^2) = g h, so z <- z (1.5 - 2 Im z^2) runs the
  iteration of App. B.1 and 4 Im z is its h;
- the arcsine step of the constant bootstrap: y (1 + y^2/6) with y = sin(theta)
  returns theta within 3 theta^5 / 40 (the next Taylor term of arcsin).
"""
import numpy as np

from oracle import cutmax_fp64 as F


def test_complex_pair_runs_the_goldschmidt_iteration():
    rng = np.random.default_rng(4)
    for _ in range(20):
        x = float(np.exp(rng.uniform(np.log(0.05), np.log(20.0))))
        y0 = float(np.sqrt(rng.uniform(0.5, 2.5) / x))
        k = int(rng.integers(2, 16))
        a = 1.5 - (y0 * y0 / 2.0) * x
        z = complex(x * y0, y0 / 8.0) * a                  # (g + i h/4) after the first step
        for _ in range(2, k + 1):
            gh = 2.0 * (z * z).imag                         # = g h
            z = z * (1.5 - gh)
        h = 4.0 * z.imag
        want = F.goldschmidt_invsqrt(x, k, y0) / 2.0        # the oracle returns 2 h
        assert abs(h - want) <= 1e-12 * abs(want)
        # and it converges to 1/(2 sqrt x) where the real iteration does
        if abs(2.0 * want * np.sqrt(x) - 1.0) < 1e-6:
            assert abs(2.0 * h * np.sqrt(x) - 1.0) < 1e-6


def test_arcsine_step_error_bound():
    theta = np.linspace(-0.4, 0.4, 4001)
    y = np.sin(theta)
    corrected = y * (1.0 + y * y / 6.0)
    bound = 3.0 * np.abs(theta) ** 5 / 40.0 + 1e-16
    assert (np.abs(corrected - theta) <= bound).all()
    # against the uncorrected reading, which errs by about theta^3 / 6: at the
    # angle of a value 1 (theta = 2 pi / 2^7 ~ 0.05) about 900 times less
    t = 2 * np.pi / 128
    assert abs(np.sin(t) - t) > 500 * abs(np.sin(t) * (1 + np.sin(t) ** 2 / 6) - t)
