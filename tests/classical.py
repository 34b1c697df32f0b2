"""Classical exact solutions used as pins that share nothing with the oracle or
the CUDA path.

Stimson & Jeffery (1926), Proc. R. Soc. A 111, 110-116: two equal rigid spheres
of radius a translating with the same velocity U along their line of centres,
centre distance d = 2a cosh(alpha) (bispherical coordinates), each feel the drag
6 pi eta a U lambda(alpha) with

  lambda = (4/3) sinh(alpha) sum_{n>=1} n(n+1) / ((2n-1)(2n+3))
           [1 - (4 sinh^2((n+1/2) alpha) - (2n+1)^2 sinh^2(alpha))
                / (2 sinh((2n+1) alpha) + (2n+1) sinh(2 alpha))].

By symmetry the two spheres under equal forces F along the line of centres move
with the same velocity F / (6 pi eta a lambda).  Far apart, the method of
reflections gives lambda = 1 - 3k/2 + 9k^2/4 + O(k^3), k = a / d (the Stokeslet
of each sphere carried by the other); at contact lambda = 0.645."""
import math


def stimson_jeffery_lambda(d_over_a):
    """Drag factor lambda of the Stimson-Jeffery series, summed until the
    terms vanish (they decay like exp(-(2n-1) alpha))."""
    alpha = math.acosh(d_over_a / 2.0)
    nmax = max(60, int(40.0 / alpha))
    sa, s2a = math.sinh(alpha), math.sinh(2.0 * alpha)
    s = 0.0
    for n in range(1, nmax + 1):
        k = 2 * n + 1
        num = 4.0 * math.sinh((n + 0.5) * alpha) ** 2 - k * k * sa * sa
        den = 2.0 * math.sinh(k * alpha) + k * s2a
        s += n * (n + 1) / ((2 * n - 1) * (2 * n + 3)) * (1.0 - num / den)
    return 4.0 / 3.0 * sa * s
