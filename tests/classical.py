"""Classical exact solutions used as pins that share nothing with the oracle or
the CUDA path: translation of two equal spheres along their line of centres in
the same direction (Stimson-Jeffery) and towards each other (Brenner), and
rotation about it (Jeffery).

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


def jeffery_torque_ratio(d_over_a, co_rotating):
    """Torque on each of two equal spheres rotating about their line of centres,
    in units of the single-sphere torque 8 pi eta a^3 Omega (Jeffery (1915),
    Proc. Lond. Math. Soc. 14, 327-338, torsional solution in bispherical
    coordinates): sinh^3(alpha) sum_{n>=1} s^(n+1) / sinh^3(n alpha) with
    s = +1 for opposite senses (the mid-plane is then a no-slip wall) and s = -1
    for the same sense.  Far apart this is 1 -/+ (a/d)^3: a rotlet of the
    neighbour turns the fluid at the sphere's centre with a^3 Omega / d^3."""
    alpha = math.acosh(d_over_a / 2.0)
    s = -1.0 if co_rotating else 1.0
    total, n = 0.0, 1
    while n * alpha < 200.0:
        total += s ** (n + 1) / math.sinh(n * alpha) ** 3
        n += 1
    return math.sinh(alpha) ** 3 * total


def approach_lambda(d_over_a):
    """Drag factor of two equal spheres approaching each other along their line
    of centres with equal and opposite velocities (each feels 6 pi eta a U
    lambda).  By symmetry the mid-plane carries no normal velocity and no shear
    stress, so this is Brenner's (1961) sphere moving normal to a plane free
    surface (Chem. Eng. Sci. 16, 242-251), with cosh(alpha) = d / 2a:

      lambda = (4/3) sinh(alpha) sum_{n>=1} n(n+1) / ((2n-1)(2n+3))
               [(4 cosh^2((n+1/2) alpha) + (2n+1)^2 sinh^2(alpha))
                / (2 sinh((2n+1) alpha) - (2n+1) sinh(2 alpha)) - 1].

    Far apart, lambda = 1 + 3k/2 + 9k^2/4 + O(k^3), k = a / d: each sphere moves
    against the Stokeslet flow of the other."""
    alpha = math.acosh(d_over_a / 2.0)
    sa, s2a = math.sinh(alpha), math.sinh(2.0 * alpha)
    s = 0.0
    for n in range(1, max(60, int(40.0 / alpha)) + 1):
        k = 2 * n + 1
        if k * alpha > 600.0:
            break
        num = 4.0 * math.cosh((n + 0.5) * alpha) ** 2 + k * k * sa * sa
        den = 2.0 * math.sinh(k * alpha) - k * s2a
        s += n * (n + 1) / ((2 * n - 1) * (2 * n + 3)) * (num / den - 1.0)
    return 4.0 / 3.0 * sa * s
