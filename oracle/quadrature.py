"""Quadrature rules of the oracle (test infrastructure only)."""
import math
import numpy as np


def gauss_legendre_01(n):
    """n-point Gauss-Legendre rule on [0, 1] (exact to degree 2n-1)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def triangle_rule(degree):
    """Collapsed Gauss-Legendre x Gauss-Legendre rule on {xi1, xi2 >= 0, xi1 + xi2 <= 1}.

    Duffy map xi1 = a (1 - b), xi2 = b with Jacobian (1 - b). With n = degree//2 + 2
    points per direction the rule is exact for total degree <= degree (the b
    direction sees degree + 1). Weights sum to 1/2. Returns (xi [n*n, 2], w [n*n]).
    """
    n = degree // 2 + 2
    a, wa = gauss_legendre_01(n)
    b, wb = gauss_legendre_01(n)
    A, B = np.meshgrid(a, b, indexing="ij")
    WA, WB = np.meshgrid(wa, wb, indexing="ij")
    xi = np.stack([(A * (1.0 - B)).ravel(), B.ravel()], axis=1)
    w = (WA * WB * (1.0 - B)).ravel()
    return xi, w


def facet_rule(k):
    """The facet rule both sides use: q = ceil((3k+1)/2) Gauss-Legendre points on [0, 1]."""
    return gauss_legendre_01(int(math.ceil((3 * k + 1) / 2.0)))
