"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these tests compares the oracle with itself: every expected value comes
from a closed form, a finite difference, a theorem of the paper's Sec. 3, a
textbook special case, brute force, or a published known-answer vector.
"""
import itertools
import math
import os

import numpy as np
import pytest

import oracle as O
from workloads import gmm_knn_graph, planted_dense, uniform_init

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rand_nonneg(g, n, r, scale=1.0):
    return g.random((n, r)) * scale


def _small_problem(n=24, r=3, seed=7):
    A, _ = planted_dense(n, r, 0.01, seed=seed)
    W = uniform_init(n, r, math.sqrt(A.mean() / r), seed=seed + 1)
    return A, W


# ---------------------------------------------------------------------------
# Philox (published known-answer vectors; Box-Muller moments)
# ---------------------------------------------------------------------------

def test_philox_known_answers(repo_root):
    path = os.path.join(repo_root, "tests", "golden", "philox4x32_10_kat.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        vals = [int(x, 16) for x in row]
        out = O.philox4x32(*[np.uint64(v) for v in vals[:6]])
        assert [int(x) for x in out] == vals[6:]


def test_philox_streams_moments():
    Z = O.philox_gaussian(300, 401, seed=12345)  # odd column count: pairs span rows
    N = Z.size
    assert abs(Z.mean()) < 5.0 / math.sqrt(N)
    assert abs(Z.var() - 1.0) < 5.0 * math.sqrt(2.0 / N)
    U = O.philox_uniform(300, 400, seed=99)
    assert U.min() > 0.0 and U.max() < 1.0
    assert abs(U.mean() - 0.5) < 5.0 / math.sqrt(12.0 * U.size)
    # distinct seeds give distinct streams
    assert not np.array_equal(O.philox_gaussian(4, 4, 1), O.philox_gaussian(4, 4, 2))


# ---------------------------------------------------------------------------
# Objectives: definition vs Frobenius expansion
# ---------------------------------------------------------------------------

def test_closed_form_objectives_match_definition():
    g = np.random.default_rng(1)
    A, W = _small_problem(30, 4, seed=3)
    Ht = _rand_nonneg(g, 30, 4)
    L = O.paper_laplacian(A)
    for gamma in (0.0, 0.3):
        fe = O.direct_objective(A, W, gamma, L, "explicit")
        fc = O.direct_objective(A, W, gamma, L, "closed")
        assert abs(fe - fc) <= 1e-12 * abs(fe)
        pe = O.penalty_objective(A, W, Ht, 0.7, gamma, L, "explicit")
        pc = O.penalty_objective(A, W, Ht, 0.7, gamma, L, "closed")
        assert abs(pe - pc) <= 1e-12 * abs(pe)
    # LAI operator: ||U E U^T||^2 = sum lam^2 enters the closed form
    U, _ = np.linalg.qr(g.normal(size=(30, 5)))
    op = O.LaiOperator(U, g.normal(size=5) * 10)
    fe = O.penalty_objective(op, W, Ht, 0.2, 0.0, None, "explicit")
    fc = O.penalty_objective(op, W, Ht, 0.2, 0.0, None, "closed")
    assert abs(fe - fc) <= 1e-12 * abs(fe)


def test_direct_objective_brute_sum():
    """1/4 sum_ij (V_ij - sum_c W_ic W_jc)^2 written with scalar loops."""
    A, W = _small_problem(6, 2, seed=11)
    s = 0.0
    for i in range(6):
        for j in range(6):
            s += (A[i, j] - sum(W[i, c] * W[j, c] for c in range(2))) ** 2
    assert abs(O.direct_objective(A, W) - 0.25 * s) <= 1e-13 * s


# ---------------------------------------------------------------------------
# Gradients: central finite differences
# ---------------------------------------------------------------------------

def _fd_check(f, grad, X, h=1e-6, tol=1e-6):
    G = grad(X)
    g = np.random.default_rng(5)
    for _ in range(6):
        E = g.normal(size=X.shape)
        d = (f(X + h * E) - f(X - h * E)) / (2 * h)
        a = float(np.sum(G * E))
        assert abs(d - a) <= tol * max(1.0, abs(a)), (d, a)


def test_gradients_finite_differences():
    g = np.random.default_rng(2)
    A, W = _small_problem(12, 3, seed=5)
    Ht = _rand_nonneg(g, 12, 3)
    Ldense = O.paper_laplacian(A)
    lam, gam = 0.4, 0.25
    _fd_check(lambda X: O.direct_objective(A, X), lambda X: O.direct_gradient(A, X), W)
    _fd_check(lambda X: O.direct_objective(A, X, gam, Ldense),
              lambda X: O.direct_gradient(A, X, gam, Ldense), W)
    _fd_check(lambda X: O.penalty_objective(A, X, Ht, lam),
              lambda X: O.penalty_grad_W(A, X, Ht, lam), W)
    _fd_check(lambda X: O.penalty_objective(A, W, X, lam, gam, Ldense),
              lambda X: O.penalty_grad_Ht(A, W, X, lam, gam, Ldense), Ht)
    U, _ = np.linalg.qr(g.normal(size=(12, 4)))
    op = O.LaiOperator(U, g.normal(size=4) * 3)
    _fd_check(lambda X: O.penalty_objective(op, X, Ht, lam),
              lambda X: O.penalty_grad_W(op, X, Ht, lam), W)
    _fd_check(lambda X: O.direct_objective(op, X), lambda X: O.direct_gradient(op, X), W)


# ---------------------------------------------------------------------------
# rho_0 and the Lipschitz bounds (Sec. 3.1-3.2)
# ---------------------------------------------------------------------------

def test_spectral_norm_against_eigensolver():
    g = np.random.default_rng(4)
    for (n, r) in [(50, 8), (200, 16), (30, 1), (64, 32)]:
        X = _rand_nonneg(g, n, r)
        G = X.T @ X
        ref = float(np.linalg.eigvalsh(G)[-1])
        assert abs(O.spectral_norm(G, 50) - ref) <= 1e-12 * ref
    assert O.spectral_norm(np.zeros((3, 3))) == 0.0


def test_lipschitz_bounds_random_pairs():
    g = np.random.default_rng(8)
    A, _ = _small_problem(20, 3, seed=9)
    Ht = _rand_nonneg(g, 20, 3)
    W = _rand_nonneg(g, 20, 3)
    lam, gam = 0.5, 0.3
    L = O.paper_laplacian(A)
    Lw = np.linalg.eigvalsh(Ht.T @ Ht)[-1] + lam
    Lh = np.linalg.eigvalsh(W.T @ W)[-1] + lam + gam * np.linalg.eigvalsh(L)[-1]
    for _ in range(20):
        X1, X2 = g.normal(size=(20, 3)), g.normal(size=(20, 3))
        d = np.linalg.norm(O.penalty_grad_W(A, X1, Ht, lam) - O.penalty_grad_W(A, X2, Ht, lam))
        assert d <= Lw * np.linalg.norm(X1 - X2) * (1 + 1e-12)
        d = np.linalg.norm(O.penalty_grad_Ht(A, W, X1, lam, gam, L) - O.penalty_grad_Ht(A, W, X2, lam, gam, L))
        assert d <= Lh * np.linalg.norm(X1 - X2) * (1 + 1e-12)


# ---------------------------------------------------------------------------
# Algorithm 1 invariants (Sec. 3.1 restatement of Li et al.)
# ---------------------------------------------------------------------------

def test_descent_lemma_and_reference_monotonicity():
    A, W = _small_problem(40, 4, seed=21)
    opts = O.Options(formulation="penalty", phi=1.0, memory=0, max_iter=15, tol=0.0)
    _, _, info = O.snmpbb_penalty(A, W, W, opts)
    nsteps = 0
    for rec in info["trace"]:
        for tr in (rec["w_trace"], rec["h_trace"]):
            prevF = math.inf
            for s in tr:
                # <grad f(Z), D_alpha(Z)> <= -(1/alpha) ||D_alpha(Z)||^2
                assert s["gd"] <= -s["dd"] / s["alpha"] + 1e-9 * max(1.0, abs(s["gd"]))
                # f(W_k) <= F_k <= F_{k-1}
                assert s["f"] <= s["F"] * (1 + 1e-13) + 1e-12
                assert s["F"] <= prevF * (1 + 1e-13) + 1e-12
                prevF = s["F"]
                assert s["beta"] > 0.0  # finite backtracking
                nsteps += 1
    assert nsteps == 15 * 2 * opts.inner_iters


def test_bb_step_within_block_curvature():
    """In a block, Y = S (H H^T + lambda I) (Sec. 3.3), so BB1 lies in
    [1/lambda_max, 1/lambda_min] of H H^T + lambda I unless clamped."""
    A, W = _small_problem(40, 4, seed=31)
    lam = 0.5
    opts = O.Options(formulation="penalty", lambda_sym=lam, max_iter=4, tol=0.0)
    Ht = W.copy()
    ev = np.linalg.eigvalsh(Ht.T @ Ht + lam * np.eye(4))
    _, _, info = O.nmpbb(lambda X: O.penalty_objective(A, X, Ht, lam),
                         lambda X: O.penalty_grad_W(A, X, Ht, lam), W,
                         lambda X: O.spectral_norm(Ht.T @ Ht), 8, opts)
    for s in info["trace"][1:]:
        assert 1.0 / ev[-1] * (1 - 1e-10) <= s["alpha"] <= 1.0 / ev[0] * (1 + 1e-10)


def test_bb2_step_within_block_curvature_and_below_bb1():
    """BB2 = <S,Y>/<Y,Y> (the least-squares step of Sec. 2.4).  In a block Y = S M with
    M = H H^T + lambda I (Sec. 3.3), so <S,Y>/<Y,Y> is a Rayleigh quotient of M^-1 taken
    at S M: it lies in [1/lambda_max(M), 1/lambda_min(M)], and by Cauchy-Schwarz it is
    at most BB1 = <S,S>/<S,Y> of the same S, Y.  S and Y are rebuilt here from the
    recorded iterates, independently of the oracle's step routine."""
    A, W = _small_problem(40, 4, seed=33)
    lam = 0.5
    opts = O.Options(formulation="penalty", lambda_sym=lam, max_iter=4, tol=0.0, bb="bb2")
    Ht = W.copy()
    M = Ht.T @ Ht + lam * np.eye(4)
    ev = np.linalg.eigvalsh(M)
    grad = lambda X: O.penalty_grad_W(A, X, Ht, lam)
    _, _, info = O.nmpbb(lambda X: O.penalty_objective(A, X, Ht, lam), grad, W,
                         lambda X: O.spectral_norm(Ht.T @ Ht), 8, opts, keep_iterates=True)
    xs = [W] + [s["X"] for s in info["trace"]]
    strictly_below = 0
    for k, s in enumerate(info["trace"][1:], start=1):
        S = xs[k] - xs[k - 1]
        Y = grad(xs[k]) - grad(xs[k - 1])
        assert np.allclose(Y, S @ M, rtol=1e-10, atol=1e-12)   # Sec. 3.3: the block is quadratic
        bb1 = np.sum(S * S) / np.sum(S * Y)
        assert 1.0 / ev[-1] * (1 - 1e-10) <= s["alpha"] <= 1.0 / ev[0] * (1 + 1e-10)
        assert s["alpha"] <= bb1 * (1 + 1e-12)
        strictly_below += s["alpha"] < bb1 * (1 - 1e-6)
    assert strictly_below >= 1  # generic S is no eigen-direction of M: BB2 < BB1 there


def test_bb_steps_equal_inverse_curvature_for_isotropic_block():
    """With H H^T + lambda I = c I (orthogonal, equal-norm columns of Ht) every BB step of
    a block is exactly 1/c, for BB1 and BB2 alike: S M = c S."""
    A, W = _small_problem(30, 3, seed=35)
    lam, c = 0.25, 2.0
    Ht = np.zeros((30, 3))
    Ht[[0, 1, 2], [0, 1, 2]] = math.sqrt(c - lam)
    for bb in ("bb1", "bb2"):
        opts = O.Options(formulation="penalty", lambda_sym=lam, max_iter=4, tol=0.0, bb=bb)
        _, _, info = O.nmpbb(lambda X: O.penalty_objective(A, X, Ht, lam),
                             lambda X: O.penalty_grad_W(A, X, Ht, lam), W,
                             lambda X: O.spectral_norm(Ht.T @ Ht), 6, opts)
        for s in info["trace"][1:]:
            assert abs(s["alpha"] - 1.0 / c) <= 1e-12, (bb, s["alpha"])


def test_naive_variant_rank_one_is_the_exact_block_recursion():
    """Naive symmetric NMPBB (Sec. 2.1, before the penalty form), r = 1, entrywise positive V:
    the W block 1/2 ||V - w h^T||^2 with h = w_k fixed has the isotropic Hessian ||h||^2 I,
    so the first Z step (rho_0 = ||h||^2) lands on its minimiser V h / ||h||^2 and D = 0
    after it.  Each outer iteration is therefore w_{k+1} = V w_k / ||w_k||^2 exactly: a
    power iteration whose direction tends to the Perron vector v_1 while the norm alternates,
    ||w_k|| ||w_{k+1}|| -> lambda_1 (c -> lambda_1 / c along v_1): the naive coupling does
    not settle, as the paper reports.  Checked against the recursion and numpy's eigensolver."""
    g = np.random.default_rng(91)
    B = g.random((30, 30))
    V = B + B.T + 1.0
    lam, U = np.linalg.eigh(V)
    v1 = np.abs(U[:, -1])
    w0 = g.random((30, 1))
    _, info = O.snmpbb_naive(V, w0, O.Options(max_iter=60, tol=0.0, memory=10), keep_iterates=True)
    ws = [w0[:, 0]] + [rec["W"][:, 0] for rec in info["trace"]]
    for k in range(1, len(ws)):
        step = V @ ws[k - 1] / float(ws[k - 1] @ ws[k - 1])
        assert np.allclose(ws[k], step, rtol=1e-10, atol=0.0), k
    w_last, w_prev = ws[-1], ws[-2]
    assert abs(float(np.linalg.norm(w_last) * np.linalg.norm(w_prev)) - lam[-1]) <= 1e-8 * lam[-1]
    assert np.allclose(w_last / np.linalg.norm(w_last), v1, atol=1e-10)


def test_naive_variant_planted_fixed_point_and_block_monotone():
    """A planted exact factor W* (V = W* W*^T) is a fixed point: its W-block gradient
    W* (W*^T W*) - V W* vanishes, so the first step leaves it in place.  From a random start,
    with phi = 1 and the eta rule, each block's reference F_k decreases (Sec. 3.1) and the
    objective 1/2 ||V - W W^T||^2 at the block ends does not increase by more than rounding."""
    g = np.random.default_rng(92)
    Ws = g.random((25, 3))
    V = Ws @ Ws.T
    W, info = O.snmpbb_naive(V, Ws, O.Options(max_iter=2, tol=0.0, memory=10))
    assert np.allclose(W, Ws, rtol=0, atol=1e-13)
    W0 = uniform_init(25, 3, math.sqrt(V.mean() / 3), seed=93)
    _, info = O.snmpbb_naive(V, W0, O.Options(max_iter=20, tol=0.0, phi=1.0, memory=0))
    for rec in info["trace"]:
        prevF = math.inf
        for s in rec["w_trace"]:
            assert s["F"] <= prevF * (1 + 1e-13) + 1e-12
            prevF = s["F"]


def test_knn_graph_on_points_of_a_line():
    """Points 0, 1, 3, 7, 15 on a line (gaps double): every point's neighbours and squared
    distances are known in closed form; S is symmetric, S_ij = exp(-d^2 / (s_i s_j)) on kNN
    pairs, the degrees are the row sums of S and A^ = D^-1/2 S D^-1/2."""
    X = np.array([[0.0], [1.0], [3.0], [7.0], [15.0]])
    nbr, d2, S, deg, A_hat = O.knn.knn_graph(X, 2, 1)
    assert nbr.tolist() == [[1, 2], [0, 2], [1, 0], [2, 1], [3, 2]]
    assert d2.tolist() == [[1, 9], [1, 4], [4, 9], [16, 36], [64, 144]]
    s = np.sqrt(d2[:, 0])  # sigma_rank = 1: distance to the nearest neighbour
    assert S[0, 1] == pytest.approx(math.exp(-1.0 / (s[0] * s[1])))
    assert S[3, 4] == pytest.approx(math.exp(-64.0 / (s[4] * s[3])))  # only 4 -> 3 is a kNN pair
    assert np.allclose(S, S.T) and S[0, 3] == 0.0 and np.all(np.diag(S) == 0.0)
    assert np.allclose(deg, S.sum(1))
    assert np.allclose(A_hat, S / np.sqrt(np.outer(deg, deg)))


def test_ari_and_accuracy_worked_example():
    """truth [0,0,0,1,1,1], pred [0,0,1,1,2,2]: table [[2,1,0],[0,1,2]]; by hand: index
    C(2,2) + C(2,2) = 2, row term C(3,2) + C(3,2) = 6, column term 3 C(2,2) = 3, C(6,2) = 15,
    expected 6 * 3 / 15 = 1.2, max (6 + 3) / 2 = 4.5, ARI = 0.8 / 3.3; best matching 0->0,
    1->2 gives accuracy 4/6.  Identical partitions up to relabelling score 1 and 1."""
    T = O.knn.contingency([0, 0, 0, 1, 1, 1], [0, 0, 1, 1, 2, 2], 2, 3)
    assert T.tolist() == [[2, 1, 0], [0, 1, 2]]
    assert O.knn.adjusted_rand_index(T) == pytest.approx(0.8 / 3.3, rel=1e-14)
    assert O.knn.matched_accuracy(T) == pytest.approx(4.0 / 6.0)
    g = np.random.default_rng(5)
    truth = g.integers(0, 4, 200)
    perm = np.array([2, 0, 3, 1])
    T2 = O.knn.contingency(truth, perm[truth], 4, 4)
    assert O.knn.adjusted_rand_index(T2) == pytest.approx(1.0) and O.knn.matched_accuracy(T2) == 1.0


def test_max_memory_reference():
    A, W = _small_problem(30, 3, seed=41)
    opts = O.Options(formulation="direct", memory=3, max_iter=12, tol=0.0)
    _, info = O.snmpbb_direct(A, W, opts)
    fs = [info["trace"][0]["f"]] + [s["f_next"] for s in info["trace"]]
    for k, s in enumerate(info["trace"]):
        if k > 0:
            assert s["F"] == max(fs[max(0, k - 2):k + 1])


# ---------------------------------------------------------------------------
# End-to-end special cases
# ---------------------------------------------------------------------------

def test_planted_exact_recovery_and_kkt():
    g = np.random.default_rng(51)
    W0 = g.random((40, 3))
    A = W0 @ W0.T
    Winit = uniform_init(40, 3, math.sqrt(A.mean() / 3), seed=52)
    opts = O.Options(formulation="direct", memory=10, max_iter=6000, tol=1e-10)
    W, info = O.snmpbb_direct(A, Winit, opts)
    assert info["residual"] <= 1e-6
    kkt = np.linalg.norm(np.minimum(W, O.direct_gradient(A, W)))
    assert kkt <= 1e-8 * info["pg0"]
    opts = O.Options(formulation="penalty", lambda_sym=1.0, max_iter=3000, tol=1e-10, objective="closed")
    W, Ht, info = O.snmpbb_penalty(A, Winit, Winit, opts)
    assert info["residual"] <= 1e-6
    assert np.linalg.norm(W - Ht) <= 1e-5 * np.linalg.norm(W)


def test_rank_one_perron_closed_form():
    """r = 1 and V entrywise positive: the minimiser of 1/4 ||V - w w^T||^2 over
    w >= 0 is sqrt(lambda_1) v_1 (Perron-Frobenius, Eckart-Young)."""
    g = np.random.default_rng(61)
    B = g.random((25, 25)) + 0.1
    V = B + B.T
    lam, vec = np.linalg.eigh(V)
    v1 = np.abs(vec[:, -1])
    w_star = math.sqrt(lam[-1]) * v1
    w0 = uniform_init(25, 1, 1.0, seed=62)
    opts = O.Options(formulation="direct", memory=10, max_iter=3000, tol=1e-12)
    w, info = O.snmpbb_direct(V, w0, opts)
    assert np.linalg.norm(w[:, 0] - w_star) <= 1e-7 * np.linalg.norm(w_star)


def test_brute_force_tiny_grid():
    """n = 4, r = 1: the converged objective is no worse than the minimum over a
    uniform grid of w >= 0, and the grid minimum is within its spacing."""
    g = np.random.default_rng(71)
    B = g.random((4, 4))
    V = B @ B.T + 0.05
    h = 0.025
    axis = np.arange(0.0, 2.0 + h / 2, h)
    best = math.inf
    for w0 in axis:
        w = np.stack(np.meshgrid(np.array([w0]), axis, axis, axis, indexing="ij"), -1).reshape(-1, 4)
        outer = w[:, :, None] * w[:, None, :]
        f = 0.25 * np.sum((V[None] - outer) ** 2, axis=(1, 2))
        best = min(best, float(f.min()))
    for seed in (72, 73):
        # start drawn as the configs draw it: U[0, sqrt(mean(V)/r)]
        w0 = uniform_init(4, 1, math.sqrt(V.mean()), seed)
        w, info = O.snmpbb_direct(V, w0, O.Options(formulation="direct", max_iter=2000, tol=1e-12))
        fconv = O.direct_objective(V, w)
        assert fconv <= best + 1e-12
        assert best - fconv <= 50 * h  # grid within a Lipschitz-times-spacing margin


def test_objective_modes_give_same_iterates():
    A, W = _small_problem(30, 3, seed=81)
    o1 = O.Options(formulation="penalty", max_iter=8, tol=0.0, objective="explicit")
    o2 = O.Options(formulation="penalty", max_iter=8, tol=0.0, objective="closed")
    W1, H1, _ = O.snmpbb_penalty(A, W, W, o1)
    W2, H2, _ = O.snmpbb_penalty(A, W, W, o2)
    assert np.linalg.norm(W1 - W2) <= 1e-10 * np.linalg.norm(W1)
    assert np.linalg.norm(H1 - H2) <= 1e-10 * np.linalg.norm(H1)


# ---------------------------------------------------------------------------
# Graph-SNMPBB (Sec. 2.2)
# ---------------------------------------------------------------------------

def test_graph_laplacian_properties_and_gamma_zero():
    A_hat, Lcsr, labels, S = gmm_knn_graph(n=300, d=8, comps=3, k=10, seed=91)
    Sd = S.to_dense()
    assert np.allclose(Sd, Sd.T)
    L = O.paper_laplacian(Sd)
    ev = np.linalg.eigvalsh(L)
    assert ev[0] >= -1e-12 and ev[-1] <= 2.0 + 1e-12
    Ld = Lcsr.to_dense()
    assert np.allclose(Ld, np.diag(Sd.sum(1)) - Sd)
    assert np.allclose(A_hat.to_dense(), Sd / np.sqrt(np.outer(Sd.sum(1), Sd.sum(1))))
    X = uniform_init(300, 3, 1.0, 92)
    assert O.inner(X, Ld @ X) >= 0.0
    Ad = A_hat.to_dense()
    W = uniform_init(300, 3, math.sqrt(Ad.mean() / 3), 93)
    a = O.snmpbb_penalty(Ad, W, W, O.Options(max_iter=5, tol=0.0, gamma=0.0), L=Ld)
    b = O.snmpbb_penalty(Ad, W, W, O.Options(max_iter=5, tol=0.0))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


# ---------------------------------------------------------------------------
# LAI-SNMPBB (Sec. 2.3, Sec. 3.3)
# ---------------------------------------------------------------------------

def test_lai_full_sketch_equals_exact():
    A, W = _small_problem(20, 3, seed=101)
    U, lam = O.lai_sketch(lambda X: A @ X, 20, 20, 0, 0, seed=102)
    op = O.LaiOperator(U, lam)
    assert np.linalg.norm(O.dense_of(op) - A) <= 1e-12 * np.linalg.norm(A)
    opts = O.Options(max_iter=6, tol=0.0)
    W1, H1, _ = O.snmpbb_penalty(A, W, W, opts)
    W2, H2, _ = O.snmpbb_penalty(op, W, W, opts)
    assert np.linalg.norm(W1 - W2) <= 1e-9 * np.linalg.norm(W1)


def test_lai_exact_low_rank_and_eigenvalues():
    g = np.random.default_rng(111)
    Q, _ = np.linalg.qr(g.normal(size=(60, 6)))
    ev = np.array([50.0, -20.0, 9.0, 4.0, -2.0, 1.0])
    V = (Q * ev) @ Q.T
    U, lam = O.lai_sketch(lambda X: V @ X, 60, 6, 4, 2, seed=112)
    assert np.allclose(np.sort(lam), np.sort(ev), rtol=1e-10, atol=1e-10)
    assert np.linalg.norm((U * lam) @ U.T - V) <= 1e-10 * np.linalg.norm(V)
    assert np.allclose(U.T @ U, np.eye(6), atol=1e-12)


def test_lai_bb_invariance_and_bias_bound():
    A, W = _small_problem(40, 3, seed=121)
    U, lam = O.lai_sketch(lambda X: A @ X, 40, 4, 2, 1, seed=122)
    op = O.LaiOperator(U, lam)
    mu = np.linalg.norm(A - O.dense_of(op))
    g = np.random.default_rng(123)
    Ht = g.random((40, 3))
    lmb = 0.3
    W1, W2 = g.random((40, 3)), g.random((40, 3))
    y_lai = O.penalty_grad_W(op, W1, Ht, lmb) - O.penalty_grad_W(op, W2, Ht, lmb)
    y_true = O.penalty_grad_W(A, W1, Ht, lmb) - O.penalty_grad_W(A, W2, Ht, lmb)
    assert np.linalg.norm(y_lai - y_true) <= 1e-12 * np.linalg.norm(y_true)
    assert np.allclose(y_true, (W1 - W2) @ (Ht.T @ Ht + lmb * np.eye(3)), rtol=1e-12, atol=1e-12)
    bias = np.linalg.norm(O.penalty_grad_W(op, W1, Ht, lmb) - O.penalty_grad_W(A, W1, Ht, lmb))
    assert bias <= mu * np.linalg.norm(Ht) * (1 + 1e-12)


def test_lambda_default_rule():
    A, _ = _small_problem(10, 2, seed=131)
    assert O.resolve_lambda(A, O.Options()) == pytest.approx(0.01 * np.linalg.norm(A), rel=1e-15)
    assert O.resolve_lambda(A, O.Options(lambda_sym=2.5)) == 2.5


# ---------------------------------------------------------------------------
# Step-controller MLP oracle: backprop vs central finite differences
# ---------------------------------------------------------------------------

def test_mlp_oracle_gradient_finite_differences():
    import oracle.mlp as M
    g = np.random.default_rng(141)
    w = g.normal(0, 0.5, M.N_PARAMS)
    phi = g.normal(0, 1, (40, M.N_IN))
    t = g.uniform(-2, 2, 40)
    grad = M.gradient(w, phi, t)
    h = 1e-6
    for idx in g.choice(M.N_PARAMS, 40, replace=False):
        e = np.zeros(M.N_PARAMS)
        e[idx] = h
        fd = (M.loss(w + e, phi, t) - M.loss(w - e, phi, t)) / (2 * h)
        assert abs(fd - grad[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, grad[idx])
    # zero weights: o = 0, multiplier 1
    assert np.allclose(M.multiplier(np.zeros(M.N_PARAMS), phi), 1.0)


def test_mlp_parameter_layout_and_multiplier_range():
    """The parameter vector follows the C ABI's documented layout W1[64][5] (row-major,
    hidden x input), b1[64], W2[64], b2: hand-built weights with a known output.  W1 routes
    input i to hidden unit i (i < 5) and hidden unit 5 + i to -input i, W2 sums them, so
    o = sum_i (relu(phi_i) + relu(-phi_i)) + b2 = sum_i |phi_i| + b2.  The multiplier
    2^(2 tanh o) lies in (1/4, 4) and is monotone in o."""
    import oracle.mlp as M
    assert (M.N_IN, M.N_HID, M.N_PARAMS) == (5, 64, 5 * 64 + 64 + 64 + 1)
    W1 = np.zeros((M.N_HID, M.N_IN))
    for i in range(M.N_IN):
        W1[i, i] = 1.0
        W1[M.N_IN + i, i] = -1.0
    b1 = np.zeros(M.N_HID)
    W2 = np.zeros(M.N_HID)
    W2[:2 * M.N_IN] = 1.0
    b2 = -0.25
    w = np.concatenate([W1.ravel(), b1, W2, [b2]])
    g = np.random.default_rng(143)
    phi = g.normal(0, 1, (30, M.N_IN))
    o, _, _ = M.forward(w, phi)
    assert np.allclose(o, np.abs(phi).sum(axis=1) + b2, rtol=0, atol=1e-14)
    m = M.multiplier(w, phi)
    assert np.all((m > 0.25) & (m < 4.0))
    order = np.argsort(o)
    assert np.all(np.diff(m[order]) >= 0)
    assert M.multiplier(w, np.zeros((1, M.N_IN)))[0] == pytest.approx(2.0 ** (2.0 * math.tanh(b2)), rel=1e-15)


def test_projected_gradient_is_the_one_sided_limit():
    """The projected gradient of min f over X >= 0 is the one-sided derivative
    lim_{t -> 0+} (X - Proj[X - t g]) / t: g where X > 0, min(g, 0) where X = 0.  Checked
    with a small step on a matrix with zero entries and gradients of both signs, and its
    norm vanishes exactly at a KKT point (X >= 0, g >= 0 on the zeros, g = 0 elsewhere)."""
    g = np.random.default_rng(144)
    X = g.random((40, 6))
    X[g.random(X.shape) < 0.4] = 0.0
    G = g.normal(0, 1, X.shape)
    t = 1e-9
    lim = (X - O.proj(X - t * G)) / t
    pos = X > 1e-6  # away from the kink at the step size used
    P = O.projected_gradient(X, G)
    assert np.allclose(P[pos], lim[pos], rtol=0, atol=1e-6)
    assert np.allclose(P[X == 0], lim[X == 0], rtol=0, atol=1e-6)
    Gk = np.where(X > 0, 0.0, np.abs(G))
    assert np.linalg.norm(O.projected_gradient(X, Gk)) == 0.0


def test_svd_init_special_cases():
    """The SVD start of Sec. 4.1 (4) on inputs whose factorization is known in closed form.
    (a) Rank one with a nonnegative vector, V = v v^T: W0 = Ht0 = v, a zero residual.
    (b) A nonnegative diagonal with distinct entries: W0 holds sqrt(d_i) e_i for the r
        largest d_i, so W0 W0^T is the best rank-r approximation (Eckart-Young) and the
        residual is sqrt(sum of the other d_i^2) / ||d||.
    (c) A symmetric matrix with a negative eigenvalue among the r largest in magnitude:
        singular values are |eigenvalues|, the absolute values remove every sign, and
        W0 = Ht0 = |Q| |lambda|^(1/2) for the eigenvectors Q."""
    g = np.random.default_rng(146)
    v = g.random(30)
    W0, Ht0 = O.svd_init(np.outer(v, v), 1)
    assert np.allclose(W0[:, 0], v, rtol=1e-12, atol=1e-14) and np.allclose(Ht0, W0, rtol=1e-12, atol=1e-14)
    d = np.array([9.0, 7.0, 5.0, 3.0, 2.0, 1.0, 0.5])
    W0, Ht0 = O.svd_init(np.diag(d), 3)
    E = np.zeros((7, 3))
    E[[0, 1, 2], [0, 1, 2]] = np.sqrt(d[:3])
    assert np.allclose(W0, E, atol=1e-14) and np.allclose(Ht0, E, atol=1e-14)
    res = np.linalg.norm(np.diag(d) - W0 @ Ht0.T) / np.linalg.norm(d)
    assert res == pytest.approx(math.sqrt(np.sum(d[3:] ** 2)) / np.linalg.norm(d), rel=1e-13)
    Q, _ = np.linalg.qr(g.normal(size=(12, 12)))
    lam = np.array([-6.0, 5.0, 4.0] + list(np.linspace(1.0, 0.1, 9)))
    V = (Q * lam) @ Q.T
    W0, Ht0 = O.svd_init(V, 3)
    ref = np.abs(Q[:, :3]) * np.sqrt(np.abs(lam[:3]))[None, :]
    assert np.allclose(W0, ref, atol=1e-12) and np.allclose(Ht0, ref, atol=1e-12)


def test_fp8_e4m3_codec_pins():
    """E4M3 from its definition: known codes, the saturation bound, round trip of every
    finite code, ties to even, the half-ulp error bound, and the tile-scale rule."""
    import oracle.fp8 as F
    assert F.decode_e4m3(0x00) == 0.0
    assert F.decode_e4m3(0x01) == 2.0 ** -9          # smallest subnormal
    assert F.decode_e4m3(0x08) == 2.0 ** -6          # smallest normal
    assert F.decode_e4m3(0x38) == 1.0
    assert F.decode_e4m3(0x7E) == 448.0              # largest finite
    assert F.decode_e4m3(0xB8) == -1.0
    assert math.isnan(F.decode_e4m3(0x7F)) and math.isnan(F.decode_e4m3(0xFF))
    vals = F.table()
    fin = np.isfinite(vals)
    assert np.sum(fin) == 254 and np.all(np.diff(vals[:0x7F]) > 0)
    codes = np.arange(256)[fin]
    expect = np.where(vals[fin] == 0, 0, codes).astype(np.uint8)   # -0 encodes as +0
    assert np.array_equal(F.encode_e4m3(vals[fin]), expect)
    # ties go to the even code: 1.0625 between 1.0 (0x38) and 1.125 (0x39) -> 1.0;
    # 1.1875 between 1.125 (0x39) and 1.25 (0x3A) -> 1.25
    assert F.encode_e4m3(np.array([1.0625, 1.1875]))[0] == 0x38
    assert F.encode_e4m3(np.array([1.0625, 1.1875]))[1] == 0x3A
    assert F.encode_e4m3(np.array([1e6]))[0] == 0x7E   # saturates
    g = np.random.default_rng(3)
    x = np.exp(g.uniform(np.log(2.0 ** -6), np.log(448.0), 10000))
    q = vals[F.encode_e4m3(x)]
    assert np.max(np.abs(q - x) / x) <= 2.0 ** -4 + 1e-15   # half an ulp of a 3-bit mantissa
    A = np.abs(g.normal(0, 3.0, (300, 260)))
    A[:128, 128:256] = 0.0                               # an all-zero tile
    codes_, S, At = F.quantize(A)
    assert S.shape == (3, 3) and S[0, 1] == 1.0
    for i in range(3):
        for j in range(3):
            m = A[i * 128:(i + 1) * 128, j * 128:(j + 1) * 128].max()
            if m > 0:
                assert 224.0 < m / S[i, j] <= 448.0 and math.log2(S[i, j]).is_integer()
    Sf = np.repeat(np.repeat(S, 128, 0), 128, 1)[:300, :260]
    normal = A / Sf >= 2.0 ** -6
    assert np.all(np.abs(At - A)[normal] <= 2.0 ** -4 * A[normal] * (1 + 1e-12))
    assert np.all(np.abs(At - A)[~normal] <= 2.0 ** -10 * Sf[~normal] * (1 + 1e-12))


def test_laplacian_norm_and_graph_block_descent():
    """gamma ||L||_2 in rho of the graph block: the power estimate sits just below the top
    eigenvalue, and the Z step of the regularised H block with that rho decreases f (a
    projected gradient step with step 1/Lipschitz), while the step without it does not have
    to (it overshoots on this graph)."""
    import oracle.snmpbb as SM
    from workloads import gmm_knn_graph
    A_hat, L, _, _ = gmm_knn_graph(n=300, d=8, comps=4, k=10, seed=91)
    Ad, Ld = A_hat.to_dense(), L.to_dense()
    lmax = np.linalg.eigvalsh(Ld)[-1]
    est = SM.laplacian_norm(Ld, 50)
    # a Rayleigh quotient never exceeds the top eigenvalue; 50 iterations get within 2%
    assert est <= lmax * (1 + 1e-12) and est >= lmax * (1 - 2e-2)
    g = np.random.default_rng(92)
    W = g.random((300, 4)) * 0.05
    Ht = g.random((300, 4)) * 0.05
    gamma, lam = 0.5, 0.01 * np.linalg.norm(Ad)
    f = lambda X: SM.penalty_objective(Ad, W, X, lam, gamma, Ld, "explicit")
    grad = SM.penalty_grad_Ht(Ad, W, Ht, lam, gamma, Ld)
    rho = np.linalg.eigvalsh(W.T @ W)[-1] + lam + gamma * lmax  # the block's Lipschitz constant
    Z = SM.proj(Ht - grad / rho)
    # sufficient decrease of a projected gradient step with step 1/Lipschitz
    assert f(Z) <= f(Ht) - 0.5 * rho * np.sum((Z - Ht) ** 2) + 1e-12 * abs(f(Ht))
