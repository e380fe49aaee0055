"""Pins of the oracle's transforms and windows against library routines and
closed forms (standard BM3D definitions: 2D DCT-II, Walsh-Hadamard along
the group, Kaiser aggregation window)."""
import numpy as np
import pytest
import scipy.fft
import scipy.linalg


def test_dct8_rows_equal_scipy_ortho_dct(oracle):
    C = oracle.dct8()
    ref = scipy.fft.dct(np.eye(8), type=2, norm="ortho", axis=0)
    np.testing.assert_allclose(C, ref, atol=1e-14)


def test_dct2d_matrix_is_kron_and_orthonormal(oracle):
    T = oracle.dct2d_matrix()
    np.testing.assert_allclose(T, np.kron(oracle.dct8(), oracle.dct8()), atol=1e-14)
    np.testing.assert_allclose(T @ T.T, np.eye(64), atol=1e-12)
    P = np.random.default_rng(1).uniform(0, 255, (8, 8))
    np.testing.assert_allclose((T @ P.ravel()).reshape(8, 8),
                               scipy.fft.dctn(P, type=2, norm="ortho"), atol=1e-10)


@pytest.mark.parametrize("n", [1, 2, 4, 8, 16, 32])
def test_hadamard_equals_scipy(oracle, n):
    np.testing.assert_allclose(oracle.hadamard(n), scipy.linalg.hadamard(n) / np.sqrt(n), atol=1e-15)


def test_hadamard_rejects_non_power_of_two(oracle):
    with pytest.raises(ValueError):
        oracle.hadamard(12)


@pytest.mark.parametrize("beta", [0.0, 2.0, 5.0])
def test_kaiser_equals_numpy(oracle, beta):
    np.testing.assert_allclose(oracle.kaiser(8, beta), np.kaiser(8, beta), atol=1e-14)


@pytest.mark.parametrize("n", [1, 2, 4, 16, 32])
def test_t3d_equals_library_composition_and_round_trips(oracle, n):
    rng = np.random.default_rng(n)
    G = rng.uniform(-50, 300, (n, 64))
    Z = oracle.t3d(G)
    # library composition: per-patch dctn, then Hadamard along the group
    D = np.stack([scipy.fft.dctn(g.reshape(8, 8), norm="ortho").ravel() for g in G])
    ref = (scipy.linalg.hadamard(n) / np.sqrt(n)) @ D
    np.testing.assert_allclose(Z, ref, atol=1e-9)
    np.testing.assert_allclose(oracle.t3d(Z, inverse=True), G, atol=1e-12 * 300)


def test_t3d_identical_patches_put_all_energy_in_row_zero(oracle):
    P = np.random.default_rng(7).uniform(0, 255, 64)
    for n in (2, 4, 8, 16, 32):
        Z = oracle.t3d(np.tile(P, (n, 1)))
        np.testing.assert_allclose(Z[0], np.sqrt(n) * scipy.fft.dctn(P.reshape(8, 8), norm="ortho").ravel(),
                                   atol=1e-9)
        assert np.abs(Z[1:]).max() < 1e-10


@pytest.mark.parametrize("L,expect", [(8, [0]), (9, [0, 1]), (11, [0, 3]), (14, [0, 3, 6]),
                                      (16, [0, 3, 6, 8])])
def test_grid_small(oracle, L, expect):
    assert list(oracle.grid(L)) == expect


@pytest.mark.parametrize("L", [8, 9, 10, 11, 37, 128, 129, 512, 1024])
def test_grid_covers_every_pixel(oracle, L):
    g = oracle.grid(L)
    cov = np.zeros(L, bool)
    for p in g:
        cov[p:p + 8] = True
    assert cov.all()
    assert g[0] == 0 and g[-1] == L - 8
    assert np.all(np.diff(g) <= 3) and np.all(np.diff(g) >= 1)
    assert len(oracle.grid(7)) == 0


def test_grid_counts_match_configured_sizes(oracle):
    assert len(oracle.grid(128)) == 41
    assert len(oracle.grid(512)) == 169
    assert len(oracle.grid(1024)) == 340


# ---- larger patch sides (the high-noise profile: 12 x 12 and 11 x 11) ----------

@pytest.mark.parametrize("k", [4, 8, 11, 12, 16])
def test_dct_k_rows_equal_scipy_ortho_dct(oracle, k):
    np.testing.assert_allclose(oracle.dct(k), scipy.fft.dct(np.eye(k), type=2, norm="ortho", axis=0), atol=1e-14)


@pytest.mark.parametrize("k", [11, 12])
def test_dct2d_matrix_k_is_kron_orthonormal_and_scipy_dctn(oracle, k):
    T = oracle.dct2d_matrix(k)
    C = oracle.dct(k)
    np.testing.assert_allclose(T, np.kron(C, C), atol=1e-14)
    np.testing.assert_allclose(T @ T.T, np.eye(k * k), atol=1e-12)
    P = np.random.default_rng(k).uniform(0, 255, (k, k))
    np.testing.assert_allclose((T @ P.ravel()).reshape(k, k), scipy.fft.dctn(P, type=2, norm="ortho"), atol=1e-10)


@pytest.mark.parametrize("k,n", [(12, 1), (12, 4), (12, 16), (11, 2), (11, 32)])
def test_t3d_k_equals_library_composition_and_round_trips(oracle, k, n):
    rng = np.random.default_rng(10 * k + n)
    G = rng.uniform(-50, 300, (n, k * k))
    Z = oracle.t3d(G)
    D = np.stack([scipy.fft.dctn(g.reshape(k, k), norm="ortho").ravel() for g in G])
    np.testing.assert_allclose(Z, (scipy.linalg.hadamard(n) / np.sqrt(n)) @ D, atol=1e-9)
    np.testing.assert_allclose(oracle.t3d(Z, inverse=True), G, atol=1e-12 * 300 * k)


@pytest.mark.parametrize("M,beta", [(11, 2.0), (12, 2.0), (12, 0.0)])
def test_kaiser_other_lengths_equal_numpy(oracle, M, beta):
    np.testing.assert_allclose(oracle.kaiser(M, beta), np.kaiser(M, beta), atol=1e-14)


@pytest.mark.parametrize("k,step", [(12, 4), (11, 6)])
@pytest.mark.parametrize("L", [12, 13, 16, 17, 37, 512, 1024])
def test_grid_k_covers_every_pixel(oracle, k, step, L):
    if L < k:
        return
    g = oracle.grid(L, k, step)
    cov = np.zeros(L, bool)
    for p in g:
        cov[p:p + k] = True
    assert cov.all() and g[0] == 0 and g[-1] == L - k
    assert np.all(np.diff(g) <= step) and np.all(np.diff(g) >= 1)
    assert len(g) == (L - k) // step + 1 + ((L - k) % step != 0)
