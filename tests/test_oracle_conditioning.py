"""The conditioning study of Sec. V A on a small cell: the condition number of the overlap matrix
(ratio of its largest to smallest eigenvalue, Γ point) of the enriched basis without
orthogonalization (EFE: the CFE block, the atomic functions' overlap and their coupling to the CFE
functions) grows quickly under mesh refinement, while that of the orthogonalized basis (OEFE: the
lumped CFE mass and M^oo, Eq. MOEFE) stays of the order of the plain CFE basis's (the lumped mass,
whose ratio of GLL weights is fixed on uniform meshes)."""
import numpy as np

from cases import oracle_problem, uniform_xb


def kappa(S):
    ev = np.linalg.eigvalsh(S)
    return ev[-1] / ev[0]


def test_orthogonalized_enrichment_keeps_the_overlap_well_conditioned():
    a = 6.0
    pos = np.array([[0.0, 0.0, 0.0], [a / 2, a / 2, a / 2]])
    k_cfe, k_efe, k_oefe = [], [], []
    for n in (2, 3, 4):   # h = 1, 2/3, 1/2 with p = 3
        pr = oracle_problem(a, uniform_xb(a, n), 3, pos, np.array([3, 4]), quad=(5, 6, 2), r0=1.5, rc=2.5)
        k_cfe.append(pr.m.max() / pr.m.min())
        k_efe.append(kappa(pr.efe_overlap_dense()))
        k_oefe.append(kappa(pr.dense_M()))
    assert np.allclose(k_cfe, k_cfe[0])                     # uniform meshes: the GLL weight ratio
    assert k_efe[0] < k_efe[1] < k_efe[2] and k_efe[2] > 10 * k_efe[0]   # EFE: fast growth (~h^-2)
    assert k_oefe[2] < 2 * k_oefe[0]                        # OEFE: slow growth
    assert k_oefe[2] < 10 * k_cfe[2] and k_efe[2] > 30 * k_oefe[2]
