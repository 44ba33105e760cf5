"""Shared helpers for the GPU parity tests (tolerances follow the stated reading).

Deposit tolerance (per entry, relative to the sum of absolute contributions):
  |G_gpu - G_ref|_e <= tol * sum_p |g_{p,e}|   and   max|G_gpu - G_ref| <= tol * max|G_ref|
with tol = 1e-12 in FP64 mode and 1e-5 in FP32 mode.  A plain relative bound per
entry is ill-posed where thermal contributions cancel.
"""
import numpy as np

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def assert_deposit_close(got, ref, ref_abs, tol, what="dG"):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    scale = np.maximum(ref_abs, np.finfo(np.float64).tiny)
    bad = err > tol * scale + 1e-300
    assert not bad.any(), (f"{what}: {bad.sum()} entries beyond {tol} * sum|contrib| "
                           f"(worst ratio {np.max(err / scale):.3e})")
    assert err.max() <= tol * max(np.abs(ref).max(), np.finfo(np.float64).tiny) + 1e-300, \
        f"{what}: max error {err.max():.3e} vs {tol} * max|ref| {np.abs(ref).max():.3e}"


def csr_tuple(m, n_cols):
    m = m.tocsr()
    m.sort_indices()
    return (m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.int8), n_cols)
