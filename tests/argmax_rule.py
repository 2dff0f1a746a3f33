"""Acceptance rule for an argmax that differs from the FP64 oracle's.

The method's precision target: IG within 1e-4 absolute + 1e-5 relative of the
oracle, read as |g - o| <= tol(o) = 1e-4 + 1e-5 |o|, and the argmax
(discretisation, partner set) equal to the oracle's except where the oracle's
top two values differ by less than that tolerance.

So a GPU argmax (d, S) other than the oracle's is accepted only if
  - the oracle's maximum o and its runner-up over every other (d, S) differ by
    at most tol(o), and
  - the oracle's IG of the GPU's (d, S) lies within tol(o) of o.
Both hold whenever the GPU evaluates every (d, S) within eps of the oracle
with 2 eps plus the float rounding of the max key below tol(o): the k = 3
tensor-core epilogue has eps <= 4.8e-5, the other paths eps below 1e-8 plus
float rounding.
"""
ATOL, RTOL = 1e-4, 1e-5


def tol(o: float) -> float:
    return ATOL + RTOL * abs(o)


def check_alternative(o: float, second: float, alt: float, what: str) -> None:
    """o: oracle maximum; second: oracle runner-up over every other choice;
    alt: oracle value of the GPU's choice."""
    t = tol(o)
    assert o - second <= t, (f"{what}: argmax differs from the oracle's, whose top two are "
                             f"{o!r} and {second!r} (gap {o - second:.3g} > tolerance {t:.3g})")
    assert o - alt <= t and alt <= o + 1e-9, (f"{what}: the GPU's choice has oracle IG {alt!r}, "
                                             f"the maximum is {o!r} (tolerance {t:.3g})")
