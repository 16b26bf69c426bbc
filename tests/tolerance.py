"""The likelihood tolerance of the parity tests.

The bar is plain relative error: |got - ref| <= rtol |ref| (1e-8 for the float64
path, 1e-5 for the mixed path).  One kind of case is measured differently: a
likelihood that is a sum of n terms of size ~log 2 pi cancelling to a total far
below them (|ref| < 0.1 n/2 log 2 pi, e.g. a 3-D squared-exponential problem whose
NLL is 22.8 from terms of ~1000).  There relative error of the total says nothing
about the arithmetic, and the bound is taken against n/2 log 2 pi instead.
"""
import math

CANCEL_FRAC = 0.1


def nll_scale(ref: float, n: int) -> float:
    """|ref|, or n/2 log 2 pi when the likelihood cancels to below a tenth of that."""
    s = 0.5 * n * math.log(2.0 * math.pi)
    return abs(ref) if abs(ref) >= CANCEL_FRAC * s else s


def nll_close(got: float, ref: float, n: int, rtol: float) -> bool:
    return abs(got - ref) <= rtol * nll_scale(ref, n)
