"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, fills documented defaults and rejects invalid arguments
before touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2606_02887_gb300.snmf as S


@pytest.fixture(scope="module")
def lib(repo_root):
    if not os.path.exists(S.LIB_PATH):
        from paper_2606_02887_gb300.build import build_library
        build_library()
    return S.load_library()


def declared_symbols(repo_root):
    txt = open(os.path.join(repo_root, "include", "snmf.h")).read()
    return sorted(set(re.findall(r"SNMF_API[^;(]*?\b(snmf_\w+)\s*\(", txt, flags=re.S)))


def test_header_symbols_exported(lib, repo_root):
    names = declared_symbols(repo_root)
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name
    assert sorted(names) == sorted(S.EXPORTED)


def test_struct_layouts_match_header(lib):
    # sizes fixed by the header's field order (LP64)
    assert C.sizeof(S.snmf_matrix) == 4 * 4 + 3 * 8 + 3 * 8 + 2 * 4 + 8
    assert C.sizeof(S.snmf_stats) == 6 * 4 + 4 * 8 + 8 + 4 * 4
    # ... tune_cache, then sym_half and branch_step
    assert C.sizeof(S.snmf_options) == 10 * 4 + 10 * 8 + 8 + 8 + 8 + 2 * 4 + 8 + 4 + 4


def test_default_options(lib):
    o = S.snmf_default_options()
    assert o.branch_step == -1 and o.step_controller == 0
    assert o.formulation == S.SNMF_PENALTY and o.precision == S.SNMF_F32 and o.sym_half == 0
    assert o.batch == 1 and o.nonmonotone_M == 10 and o.max_ls == 20 and o.inner_iters == 5
    assert o.theta == 1e-3 and o.phi == 1.7 and o.tol == 1e-4 and o.lambda_sym < 0
    assert o.alpha_min == 1e-10 and o.alpha_max == 1e10 and o.direct_rho_factor == 3.0


def _create(lib, m, r, o):
    h = C.c_void_p()
    st = lib.snmf_create(C.byref(h), C.byref(m), r, C.byref(o), None)
    return st, h


def test_invalid_arguments_rejected_before_launch(lib):
    A = np.eye(8)
    m, _ = S.dense_matrix(A)
    o = S.snmf_default_options()
    assert _create(lib, m, 0, o)[0] == S.SNMF_ERR_ARG            # r < 1
    m0, _ = S.dense_matrix(A)
    m0.n = 0                                                     # empty matrix
    assert _create(lib, m0, 1, o)[0] == S.SNMF_ERR_ARG
    assert _create(lib, m, 9, o)[0] == S.SNMF_ERR_ARG            # r > n
    assert _create(lib, m, 300, o)[0] == S.SNMF_ERR_ARG          # r > 256
    bad = S.snmf_default_options(batch=0)
    assert _create(lib, m, 2, bad)[0] == S.SNMF_ERR_ARG
    bad = S.snmf_default_options(theta=1.5)
    assert _create(lib, m, 2, bad)[0] == S.SNMF_ERR_ARG
    bad = S.snmf_default_options(nonmonotone_M=65)
    assert _create(lib, m, 2, bad)[0] == S.SNMF_ERR_ARG
    bad = S.snmf_default_options(step_controller=4, batch=8)     # rollout groups of 9 restarts
    assert _create(lib, m, 2, bad)[0] == S.SNMF_ERR_ARG
    bad = S.snmf_default_options(step_controller=5)
    assert _create(lib, m, 2, bad)[0] == S.SNMF_ERR_ARG
    m2, _ = S.dense_matrix(A)
    m2.ld = 4                                                    # ld < n
    assert _create(lib, m2, 2, o)[0] == S.SNMF_ERR_ARG
    m3, _ = S.dense_matrix(A)
    m3.kind = 7
    assert _create(lib, m3, 2, o)[0] == S.SNMF_ERR_ARG
    msg = lib.snmf_last_error(None).decode()
    assert "kind" in msg
    assert lib.snmf_destroy(None) == S.SNMF_OK


def test_no_cpu_fallback_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    A = np.eye(8)
    st, h = _create(lib, S.dense_matrix(A)[0], 2, S.snmf_default_options())
    assert st == S.SNMF_ERR_CUDA and not h.value


def test_noalloc_limits_follow_the_header(lib, repo_root):
    """The allocation-free product's published limits: the binding's constants equal the
    header's macros, n = SNMF_NOALLOC_MAX_ROWS + 64 and an oversized slice pair are rejected
    with SNMF_ERR_ARG before any CUDA call, and n = SNMF_NOALLOC_MAX_ROWS passes the size
    checks (without a GPU the call then fails with SNMF_ERR_CUDA; it is not run where a GPU
    is present, because the pointers here are placeholders)."""
    txt = open(os.path.join(repo_root, "include", "snmf.h")).read()
    macros = dict(re.findall(r"#define (SNMF_NOALLOC_\w+) (.+)", txt))
    env = {}
    for name, expr in macros.items():
        e = expr.replace("ull", "").replace("ll", "").replace("(int64_t)", "")
        for k, v in env.items():
            e = e.replace(k, str(v))
        env[name] = int(eval(e, {}, {}))
    assert env["SNMF_NOALLOC_SCRATCH_BYTES"] == S.NOALLOC_SCRATCH_BYTES
    assert env["SNMF_NOALLOC_MAX_SLICE_PAIR_BYTES"] == S.NOALLOC_MAX_SLICE_PAIR_BYTES
    assert env["SNMF_NOALLOC_MAX_ROWS"] == S.NOALLOC_MAX_ROWS == 1048512
    fake = C.c_void_p(0x1000)
    out = C.c_double()
    f = lib.snmf_apply_dense_noalloc
    n_max = S.NOALLOC_MAX_ROWS
    assert f(fake, S.SNMF_F32, n_max + 64, n_max + 64, fake, fake, 1, C.byref(out), None) == S.SNMF_ERR_ARG
    cols = S.NOALLOC_MAX_SLICE_PAIR_BYTES // (2 * 4096 * 4) + 1
    assert f(fake, S.SNMF_F32, 4096, 4096, fake, fake, cols, C.byref(out), None) == S.SNMF_ERR_ARG
    assert f(fake, 7, 64, 64, fake, fake, 1, C.byref(out), None) == S.SNMF_ERR_ARG
    assert f(fake, S.SNMF_F32, 64, 32, fake, fake, 1, C.byref(out), None) == S.SNMF_ERR_ARG
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present: placeholder pointers must not reach a launch")
    assert f(fake, S.SNMF_F32, n_max, n_max, fake, fake, 1, C.byref(out), None) == S.SNMF_ERR_CUDA


def test_rollout_labels_pick_the_lowest_objective_and_break_ties_to_one():
    from paper_2606_02887_gb300.train_controller import rollout_labels
    f = np.array([[5.0, 4.0, 3.0, 2.5, 2.0, 2.2, 1.0, 3.0, 9.0],    # candidate 6: multiplier 2
                  [1.0] * 9,                                          # all equal: plain step
                  [2.0, 2.0, 2.0, 2.0, 1.0, 1.0 - 1e-15, 2, 2, 2],  # within the tie margin
                  [0.5, 1, 1, 1, 1, 1, 1, 1, 1],                      # multiplier 1/4
                  [np.nan, 1, 1, 1, 1, 1, 1, 1, 1]])                  # non-finite: dropped
    lab = rollout_labels(f)
    assert lab[:4].tolist() == [1.0, 0.0, 0.0, -2.0] and np.isnan(lab[4])


def test_rollout_targets_score_by_objective_or_projected_gradient():
    from paper_2606_02887_gb300.train_controller import rollout_targets
    feats = np.arange(15, dtype=np.float32).reshape(3, 5)
    fv = np.array([[3.0, 2, 1, 2, 2, 2, 2, 2, 2],       # objective: multiplier 2^-1
                   [1.0] * 9,
                   [np.inf, 1, 1, 1, 1, 1, 1, 1, 1]])     # dropped
    pv = np.array([[1.0, 1, 1, 1, 1, 1, 1, 1, 0.5],     # projected gradient: multiplier 4
                   [1.0, 1, 1, 1, 1, 0.9, 1, 1, 1],      # 10% better: kept at margin 0.05 only
                   [1.0] * 9])
    f, t = rollout_targets(feats, fv, pv, score="f")
    assert f.shape == (2, 5) and t.tolist() == [-1.0, 0.0] and np.array_equal(f, feats[:2])
    f, t = rollout_targets(feats, fv, pv, score="pg", margin=0.05)
    assert t.tolist() == [2.0, 0.5, 0.0]
    f, t = rollout_targets(feats, fv, pv, score="pg", margin=0.2)
    assert t.tolist() == [2.0, 0.0, 0.0]
