"""Shared test utilities: move generator output to the GPU and run the oracle
on the same arrays.  No arithmetic of the method lives here."""
import numpy as np
import pytest


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2008_01440_gb300.build import build
    build()
    return torch


def to_dev(torch, a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.cuda()


def csr_to_gpu(torch, nc, A):
    """Upload a workloads.CSR and wrap it in an nc_matrix handle."""
    rp = to_dev(torch, A.rowptr)
    cl = to_dev(torch, A.col)
    vl = to_dev(torch, A.val)
    return nc.nc_matrix_csr(rp, cl, vl)


def rel_err(got, ref):
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def elem_err(got, ref):
    """max_i |got_i - ref_i| / max_i |ref_i|"""
    got = np.asarray(got)
    ref = np.asarray(ref)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


def gershgorin_np(rowptr, col, val, n):
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    s = np.zeros(n)
    np.add.at(s, rows, np.abs(val))
    return float(s.max())
