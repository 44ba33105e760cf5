"""Shared helpers for the GPU parity tests (tolerances follow the stated reading).

Deposit tolerance (per entry, relative to the sum of absolute contributions):
  |G_gpu - G_ref|_e <= tol * sum_p |g_{p,e}|   and   max|G_gpu - G_ref| <= tol * max|G_ref|
with tol = 1e-12 in FP64 mode and 1e-5 in FP32 mode.  A plain relative bound per
entry is ill-posed where thermal contributions cancel.
"""
import numpy as np

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def fp32_continuity_tol(n_particles, n_nodes, n_edges):
    """Relative bound on the FP32 continuity residual |D0^T dG - dQ| against the node scale.

    The deposits are FP32 sums of k terms each (k ~ 4 N_p / N_n per node charge, 6 N_p / N_e
    per edge current); their rounding grows like sqrt(k) * 2^-24 for independent roundings.
    The bound takes 8 times that, and never less than 1e-6.
    """
    k = max(4.0 * n_particles / n_nodes, 6.0 * n_particles / n_edges, 1.0)
    return max(1e-6, 8.0 * 2.0 ** -24 * k ** 0.5)


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
