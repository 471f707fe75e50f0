"""1D rules and the Lagrange basis of spectral finite elements (Sec. III A).

Spectral elements use Lagrange polynomials on Gauss-Lobatto-Legendre (GLL)
nodes; with GLL quadrature the nodes and the quadrature points coincide and
the CFE overlap matrix becomes diagonal (Sec. III A, discussion of Eq. orthCGLL).
"""
import numpy as np
from numpy.polynomial import legendre as L


def gll(p):
    """GLL nodes (ascending, including -1 and 1) and weights for order p.

    Nodes: -1, 1 and the roots of P_p'. Weights: 2 / (p (p+1) P_p(x)^2).
    """
    if p < 1:
        raise ValueError("p >= 1")
    cp = np.zeros(p + 1)
    cp[p] = 1.0
    inner = np.sort(np.real(L.legroots(L.legder(cp)))) if p > 1 else np.array([])
    x = np.concatenate([[-1.0], inner, [1.0]])
    Pp = L.legval(x, cp)
    w = 2.0 / (p * (p + 1) * Pp ** 2)
    return x, w


def gauss(n):
    """n-point Gauss-Legendre rule on [-1, 1] (library routine)."""
    return L.leggauss(n)


def lagrange(nodes, x):
    """Values and derivatives of the Lagrange polynomials on ``nodes`` at ``x``.

    Returns (V, D), each of shape (len(x), len(nodes)):
    V[q, a] = L_a(x_q), D[q, a] = L_a'(x_q). Plain product formula.
    """
    nodes = np.asarray(nodes, float)
    x = np.atleast_1d(np.asarray(x, float))
    n = len(nodes)
    V = np.ones((len(x), n))
    D = np.zeros((len(x), n))
    for a in range(n):
        for b in range(n):
            if b == a:
                continue
            V[:, a] *= (x - nodes[b]) / (nodes[a] - nodes[b])
        for c in range(n):
            if c == a:
                continue
            term = np.full(len(x), 1.0 / (nodes[a] - nodes[c]))
            for b in range(n):
                if b == a or b == c:
                    continue
                term *= (x - nodes[b]) / (nodes[a] - nodes[b])
            D[:, a] += term
    return V, D
