"""Graph-SNMPBB with the paper's own Laplacian L = I - D^-1/2 A D^-1/2 (Sec. 2.2, Eq. (5)),
selected by snmf_set_graph_reg(h, NULL, gamma): the FP64 iterates follow the oracle, which
forms that L densely from A by its definition (oracle.paper_laplacian)."""
import math

import numpy as np
import pytest

import oracle as O
import paper_2606_02887_gb300.snmf as S
from workloads import gmm_knn_graph, planted_dense, uniform_init

from gpu_helpers import gpu_solve, rel
from test_gpu_parity import ITER_TOL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def knn():
    A_hat, _, labels, _ = gmm_knn_graph(n=400, d=8, comps=4, k=10, seed=65)
    return A_hat, A_hat.to_dense(), labels


def test_paper_laplacian_penalty_fp64_csr(knn):
    A_hat, Ad, _ = knn
    r = 4
    W0 = uniform_init(400, r, math.sqrt(Ad.mean() / r), seed=66)
    Lp = O.paper_laplacian(Ad)
    csr = (A_hat.rowptr, A_hat.colidx, A_hat.values)
    for gamma in (0.1, 1.0):
        opts = O.Options(max_iter=8, tol=0.0, gamma=gamma, memory=10, objective="closed")
        Wo, Ho, _ = O.snmpbb_penalty(Ad, W0, W0, opts, L=Lp)
        W, H, _, _, _ = gpu_solve(None, W0, r, W0, csr=csr, L="paper", gamma=gamma, max_iter=8, tol=0.0)
        assert rel(W, Wo) <= ITER_TOL and rel(H, Ho) <= ITER_TOL, gamma


def test_paper_laplacian_dense_penalty_and_direct_fp64():
    """Dense A (a planted problem with a row of zeros: a node of degree 0 gets scaling 0), the
    penalty form and the direct form, against the oracle's dense L."""
    A, _ = planted_dense(200, 3, 0.01, seed=67)
    A[5, :] = 0.0
    A[:, 5] = 0.0
    r = 3
    W0 = uniform_init(200, r, math.sqrt(A.mean() / r), seed=68)
    Lp = O.paper_laplacian(A)
    assert np.allclose(Lp[5], np.eye(200)[5])
    gamma = 0.2 * float(np.linalg.norm(A)) / 200
    opts = O.Options(max_iter=6, tol=0.0, gamma=gamma, memory=10, objective="closed")
    Wo, Ho, _ = O.snmpbb_penalty(A, W0, W0, opts, L=Lp)
    W, H, _, _, _ = gpu_solve(A, W0, r, W0, L="paper", gamma=gamma, max_iter=6, tol=0.0)
    assert rel(W, Wo) <= ITER_TOL and rel(H, Ho) <= ITER_TOL
    od = O.Options(formulation="direct", gamma=gamma, max_iter=10, tol=0.0, memory=10, objective="closed")
    Wd, _ = O.snmpbb_direct(A, W0, od, L=Lp)
    W, _, _, _, _ = gpu_solve(A, W0, r, L="paper", gamma=gamma, formulation=S.SNMF_DIRECT, max_iter=10, tol=0.0)
    assert rel(W, Wd) <= ITER_TOL


def test_paper_laplacian_fp32_clustering(knn):
    """FP32, 8 restarts to tolerance 1e-4: the best restart's clustering (argmax of Ht rows)
    recovers the 4 planted components, and its residual is within 1e-3 of the oracle's."""
    A_hat, Ad, labels = knn
    r, b = 4, 8
    Ws = [uniform_init(400, r, math.sqrt(Ad.mean() / r), seed=70 + j) for j in range(b)]
    csr = (A_hat.rowptr, A_hat.colidx, A_hat.values)
    W, H, st, stats, per = gpu_solve(None, np.concatenate(Ws, 1), r, np.concatenate(Ws, 1),
                                     precision=S.SNMF_F32, csr=csr, L="paper", gamma=0.1, batch=b,
                                     max_iter=500, tol=1e-4)
    assert st == S.SNMF_OK, stats
    best = int(np.argmin(per["f"]))
    Wo, Ho, info = O.snmpbb_penalty(Ad, Ws[best], Ws[best], O.Options(max_iter=500, tol=1e-4, gamma=0.1, memory=10,
                                                                     objective="closed"), L=O.paper_laplacian(Ad))
    res = float(np.linalg.norm(Ad - W[:, best * r:(best + 1) * r] @ H[:, best * r:(best + 1) * r].T)
                / np.linalg.norm(Ad))
    assert abs(res - info["residual"]) <= 1e-3, (res, info["residual"])
    pred = np.argmax(H[:, best * r:(best + 1) * r], axis=1)
    # best one-to-one matching of 4 clusters by brute force over the 24 permutations
    import itertools
    acc = max(np.mean(np.asarray(p)[pred] == labels) for p in itertools.permutations(range(r)))
    assert acc >= 0.95, acc
