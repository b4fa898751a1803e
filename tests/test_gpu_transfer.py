"""Transfer-matrix spectrum of the environment (ctm_transfer_spectrum, Sec. II.C, Eq. 3)
against the FP64 CPU oracle (dense LAPACK eigenvalues, or ARPACK on the oracle's
matrix-free apply), on the same environment; and the exact-Ising pin through the
CUDA path.

Tolerances: the iteration stops when the leading normalised magnitudes change by
less than 1e-12 between checks; both sides are FP64 (the split engine's
truncation, ~1e-12 relative, in split mode), so lambda_i agree to 1e-9.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2509_05090_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctm(A, chi, **kw):
    from paper_2509_05090_gb300 import binding
    return binding.CTM(A, chi, **kw)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("split_bf16", 1e-9)])
def test_transfer_spectrum_matches_oracle_ising(ctm_lib, prec, tol):
    ref = O.OracleCTM(I.ising_site_tensor(0.3), 16)
    ref.converge(1000, 1e-13)
    lam_ref, xi_ref, gap_ref = ref.transfer_spectrum(nev=4)
    g = _ctm(I.ising_site_tensor(0.3), 16, precision=prec, n_split=5)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    lam, xi, gap, iters, ok = g.ctm_transfer_spectrum(nev=4)
    assert ok
    assert np.max(np.abs(lam - lam_ref)) <= tol
    assert abs(xi - xi_ref) <= 10 * tol * xi_ref and abs(gap - gap_ref) <= 1e-6 * abs(gap_ref)
    g.close()


def test_transfer_spectrum_matches_oracle_random_d4(ctm_lib):
    """Random D = 4, chi = 32 environment (after 5 oracle steps); transfer matrix of
    dimension 16384: ARPACK on the oracle side."""
    w = I.WORKLOADS["kitaev_D4_chi32"]
    ref = O.OracleCTM(w.site_tensor(), w.chi)
    for _ in range(5):
        ref.step()
    O.set_threads(0)
    lam_ref, xi_ref, gap_ref = ref.transfer_spectrum(nev=3)
    g = _ctm(w.site_tensor(), w.chi)
    g.ctm_set_env(ref.C, ref.T, ref.Q)
    lam, xi, gap, iters, ok = g.ctm_transfer_spectrum(nev=3)
    assert ok
    assert np.max(np.abs(lam - lam_ref)) <= 1e-9
    g.close()


def test_transfer_spectrum_extrapolates_to_exact_ising_xi(ctm_lib):
    """The Sec. II.C extrapolation xi^-1(chi) = xi^-1(inf) + a ln(lambda_1/lambda_2) over
    chi = 16, 24 of the GPU spectra reproduces the exact honeycomb Ising correlation
    length along the Bravais direction (beta = 0.3)."""
    from test_oracle_pins import _ising_xi_along_chains
    exact = _ising_xi_along_chains(0.3)
    res = []
    for chi in (16, 24):
        g = _ctm(I.ising_site_tensor(0.3), chi)
        g.ctm_converge(max_steps=1000, tol=1e-13)
        lam, xi, gap, iters, ok = g.ctm_transfer_spectrum(nev=3)
        assert ok
        res.append((xi, gap))
        g.close()
    (x1, g1), (x2, g2) = res
    slope = (1 / x1 - 1 / x2) / (g1 - g2)
    xi_inf = 1.0 / (1 / x2 - slope * g2)
    assert x1 < x2 < exact
    assert abs(xi_inf - exact) < 1e-4 * exact


def test_transfer_spectrum_benchmark_size(ctm_lib):
    """D = 6, chi = 72 converging near-product state (transfer matrix of dimension
    186624).  Below lambda_0 = 1 its spectrum is a dense cluster of order eps^2 ~ 6e-6
    (every one-bond excitation of the product state), which a subspace of 8 vectors
    does not resolve into lambda_1, lambda_2 -- so no convergence is required here; after
    200 iterations the two precisions agree on the leading magnitudes and on xi."""
    w = I.WORKLOADS["kh_D6_chi72_conv"]
    out = []
    for prec in ("fp64", "split_bf16"):
        g = _ctm(w.site_tensor(), w.chi, precision=prec, n_split=5)
        g.ctm_converge(max_steps=w.steps, tol=w.tol)
        lam, xi, gap, iters, ok = g.ctm_transfer_spectrum(nev=3, max_iter=200)
        assert lam[0] == 1.0 and 0.0 < lam[2] <= lam[1] < 1e-4
        out.append((lam, xi))
        g.close()
    assert np.max(np.abs(out[0][0] - out[1][0])) <= 1e-9
    assert abs(out[0][1] - out[1][1]) <= 1e-6 * out[0][1]
