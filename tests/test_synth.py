"""The seeded input generators: shapes, determinism and the properties the
method relies on (M symmetric positive definite with unit diagonal)."""
import numpy as np

from paper_1210_7325_gb300 import synth


def test_kinship_spd_unit_diagonal():
    M = synth.kinship_M(120, 0.4, seed=1, n_markers=300)
    assert M.shape == (120, 120)
    assert np.array_equal(M, M.T)
    assert np.allclose(np.diag(M), 1.0)
    w = np.linalg.eigvalsh(M)
    assert w.min() >= 0.6 - 1e-12  # (1 - h) is a lower bound of the spectrum
    # rank-deficient kinship (markers < n) leaves eigenvalue 1 - h in the spectrum
    M2 = synth.kinship_M(80, 0.5, seed=2, n_markers=40)
    assert abs(np.linalg.eigvalsh(M2).min() - 0.5) < 1e-10


def test_determinism_and_streams():
    a = synth.problem(50, 4, 10, 0.4, seed=7, n_markers=60)
    b = synth.problem(50, 4, 10, 0.4, seed=7, n_markers=60)
    for key in a:
        assert np.array_equal(a[key], b[key])
    c = synth.problem(50, 4, 10, 0.4, seed=8, n_markers=60)
    assert not np.array_equal(a["XR"], c["XR"])


def test_covariates_and_genotypes():
    XL = synth.covariates(30, 4, seed=3)
    assert XL.shape == (30, 3) and XL.flags.f_contiguous
    assert np.all(XL[:, 0] == 1.0)
    assert synth.covariates(30, 1, seed=3).shape == (30, 0)
    XR = synth.genotypes_np(200, 20, seed=4)
    assert XR.dtype == np.int8 and XR.flags.f_contiguous
    assert set(np.unique(XR)).issubset({0, 1, 2})
    T = synth.genotypes_torch(64, 33, seed=5, chunk=10).numpy()
    assert T.shape == (33, 64) and set(np.unique(T)).issubset({0, 1, 2})
    T2 = synth.genotypes_torch(64, 33, seed=5, chunk=10).numpy()
    assert np.array_equal(T, T2)
