"""Builders of small seeded problems shared by the tests (oracle side)."""
import math

import numpy as np

import workloads as W
from oracle.enrichment import Enrichment
from oracle.mesh import Mesh
from oracle.operators import Problem
from oracle.quadrature import Quadrature


def oracle_problem(a, xb, p, pos, Z, k=(0.0, 0.0, 0.0), quad=None, orbitals=W.ORBITALS_1S_2P,
                   r0=3.0, rc=4.0, ngrid=2000, enrich=True):
    """An oracle Problem; ``quad`` = (nq_cell, nq_enr, depth)."""
    mesh = Mesh(a, xb, p)
    nq_cell, nq_enr, depth = quad or (p + 1, p + 3, 4)
    pos = np.asarray(pos, float).reshape(-1, 3)
    Z = np.asarray(Z, int)
    q = Quadrature(mesh, pos if enrich else np.zeros((0, 3)), rc, nq_cell, nq_enr, depth)
    if enrich and len(Z):
        R, dR = W.radial_tables(Z, orbitals, rc=rc, ngrid=ngrid)
        enr = Enrichment(a, pos, W.orbital_lm_codes(orbitals), R, dR, r0, rc)
    else:
        enr = Enrichment(a, np.zeros((0, 3)), np.zeros(0, int), np.zeros((0, 0, ngrid)),
                         np.zeros((0, 0, ngrid)), r0, rc)
    return Problem(mesh, q, enr, k)


def uniform_xb(a, n):
    return np.stack([np.linspace(0.0, a, n + 1)] * 3)


def small_case(k=(0.0, 0.0, 0.0), n=2, p=3, a=6.0, quad=(4, 5, 2), seed=0):
    """Two atoms (Z = 3, 4) in a small periodic box: several cells, enrichment on."""
    pos = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]])
    Z = np.array([3, 4])
    pr = oracle_problem(a, uniform_xb(a, n), p, pos, Z, k=k, quad=quad, r0=1.5, rc=2.5)
    V = W.veff(pr.quad.points, a, pos, Z, sigma=0.3)
    pr.build(V)
    return pr, V


def switched_coulomb(points, a, R, Z, r1=4.5, r2=5.0):
    """-Z/r on the minimal image, smoothly switched to 0 between r1 and r2."""
    d = np.asarray(points) - R
    d -= a * np.round(d / a)
    r = np.sqrt(np.sum(d * d, 1))
    t = np.clip((r - r1) / (r2 - r1), 0.0, 1.0)
    s = 1.0 - t * t * (3 - 2 * t)
    return -Z / np.maximum(r, 1e-300) * s
