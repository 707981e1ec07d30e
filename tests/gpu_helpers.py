"""Helpers shared by the GPU tests: run the library through the C ABI on torch
device buffers and return numpy results."""
from __future__ import annotations

import numpy as np

import paper_2606_02887_gb300.snmf as S


def torch_dev():
    import torch
    return torch, torch.device("cuda:0")


def gpu_solve(A, W0, r, Ht0=None, precision=S.SNMF_F64, csr=None, L=None, gamma=0.0,
              lai=None, host=False, **opt):
    """Solve with the library.  A: dense numpy (or None with csr=(rowptr, colidx, vals)).
    L: an explicit CSR triple, or "paper" for the normalized Laplacian of A (L == NULL).
    Returns (W, Ht, status, stats, per-restart stats)."""
    torch, dev = torch_dev()
    tdt = torch.float64 if precision == S.SNMF_F64 else torch.float32
    keep = []
    if csr is not None:
        rp, ci, va = csr
        rp_t = torch.tensor(rp, dtype=torch.int32, device=dev)
        ci_t = torch.tensor(ci, dtype=torch.int32, device=dev)
        va_t = torch.tensor(va, dtype=tdt, device=dev)
        m = S.csr_matrix(len(rp) - 1, rp_t, ci_t, va_t)
        keep += [rp_t, ci_t, va_t]
    else:
        At = torch.tensor(A, dtype=tdt, device=dev)
        m = S.dense_matrix(At)
        keep.append(At)
    o = S.snmf_default_options(precision=precision, **opt)
    h = S.snmf_create(m, r, o)
    try:
        if isinstance(L, str) and L == "paper":
            S.snmf_set_graph_reg(h, None, gamma)  # L = I - D^-1/2 A D^-1/2 of the handle's A
        elif L is not None:
            lrp, lci, lva = L
            lt = (torch.tensor(lrp, dtype=torch.int32, device=dev),
                  torch.tensor(lci, dtype=torch.int32, device=dev),
                  torch.tensor(lva, dtype=tdt, device=dev))
            keep.append(lt)
            S.snmf_set_graph_reg(h, S.csr_matrix(len(lrp) - 1, *lt), gamma)
        if lai is not None:
            S.snmf_lai_sketch(h, *lai)
        if host:
            W = np.array(W0, dtype=np.float64 if precision == S.SNMF_F64 else np.float32, copy=True)
            H = None if Ht0 is None else np.array(Ht0, dtype=W.dtype, copy=True)
            st, stats = S.snmf_solve_host(h, W, H)
            Wn, Hn = W, H
        else:
            W = None if W0 is None else torch.tensor(W0, dtype=tdt, device=dev)
            H = None if Ht0 is None else torch.tensor(Ht0, dtype=tdt, device=dev)
            st, stats = S.snmf_solve(h, W, H)
            if W is None:
                W = torch.empty((A.shape[0] if A is not None else len(csr[0]) - 1, r * o.batch),
                                dtype=tdt, device=dev)
                H = torch.empty_like(W)
                S.snmf_get_factors(h, W, H)
            torch.cuda.synchronize()
            Wn = W.cpu().numpy().astype(np.float64)
            Hn = None if H is None else H.cpu().numpy().astype(np.float64)
        per = S.snmf_restart_stats(h, o.batch)
    finally:
        S.snmf_destroy(h)
    return Wn, Hn, st, stats, per


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
