"""The host QR step of the spectrum call (ssd_hessenberg_eigenvalues) on the
CPU, no GPU needed: exact results where the Hessenberg structure fixes them
(deflated and triangular matrices, the 2 x 2 closed form, companion matrices
of known roots), backward error of every eigenvalue, trace and determinant,
clustered spectra like the D-N iteration matrix's, conjugate-pair layout,
leading blocks of an (m+1) x m Arnoldi matrix, and invalid arguments."""
import ctypes

import numpy as np
import pytest

SSD_EINVAL = 1


@pytest.fixture(scope="module")
def ssd():
    from paper_2110_10749_gb300 import build
    build.build()
    import paper_2110_10749_gb300 as m
    m.lib()
    return m


def hessenberg(rng, n, scale=1.0):
    return np.triu(rng.normal(size=(n, n)) * scale, -1)


def backward_errors(H, lam):
    nrm = np.linalg.norm(H, 2)
    n = H.shape[0]
    return np.array([np.linalg.svd(H - l * np.eye(n), compute_uv=False)[-1] / nrm for l in lam])


def reduce_to_hessenberg(A):
    """Householder reduction (orthogonal similarity) written out here."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    for k in range(n - 2):
        x = A[k + 1:, k].copy()
        a = np.linalg.norm(x)
        if a == 0.0:
            continue
        v = x.copy()
        v[0] += np.copysign(a, x[0])
        v /= np.linalg.norm(v)
        A[k + 1:, :] -= 2.0 * np.outer(v, v @ A[k + 1:, :])
        A[:, k + 1:] -= 2.0 * np.outer(A[:, k + 1:] @ v, v)
    return np.triu(A, -1)


def random_orthogonal(rng, n):
    q, r = np.linalg.qr(rng.normal(size=(n, n)))
    return q * np.sign(np.diag(r))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 10, 40, 120])
def test_random_hessenberg_backward_error_trace_det(ssd, n):
    rng = np.random.default_rng(100 + n)
    H = hessenberg(rng, n)
    lam = ssd.hessenberg_eigenvalues(H)
    assert lam.shape == (n,)
    assert backward_errors(H, lam).max() < 1e-12
    assert abs(lam.sum() - np.trace(H)) < 1e-12 * n * np.abs(H).max()
    # conjugate pairs come in adjacent entries, positive imaginary part first
    i = 0
    while i < n:
        if lam[i].imag != 0.0:
            assert lam[i].imag > 0 and lam[i + 1] == np.conj(lam[i])
            i += 2
        else:
            i += 1
    if n <= 10:
        sign, logdet = np.linalg.slogdet(H)
        prod = np.prod(lam)
        assert abs(prod - sign * np.exp(logdet)) < 1e-10 * max(1.0, abs(prod))


def test_triangular_matrix_deflates_to_its_diagonal_exactly(ssd):
    rng = np.random.default_rng(3)
    H = np.triu(rng.normal(size=(12, 12)))
    lam = ssd.hessenberg_eigenvalues(H)
    assert np.array_equal(lam.real, np.diag(H)) and not lam.imag.any()


def test_two_by_two_closed_form(ssd):
    for p, q, r, t in ((1.0, 2.0, 3.0, 4.0), (0.3, -2.0, 1.5, 0.1), (2.0, 1.0, 0.0, 2.0), (0.0, 1.0, -1.0, 0.0)):
        lam = ssd.hessenberg_eigenvalues([[p, q], [r, t]])
        m, d = 0.5 * (p + t), 0.5 * (p - t)
        disc = d * d + q * r
        ref = [m + np.sqrt(disc + 0j), m - np.sqrt(disc + 0j)]
        assert sorted(lam, key=lambda z: (z.real, z.imag)) == pytest.approx(
            sorted(ref, key=lambda z: (z.real, z.imag)), abs=1e-15)


@pytest.mark.parametrize("roots", [[1.0, -1.0, 2.0, -2.0, 3.0, 0.5], [0.25, 0.5, 0.75, 1.0]])
def test_companion_matrix_gives_the_polynomial_roots(ssd, roots):
    c = np.poly(roots)                       # monic coefficients, highest power first
    n = len(roots)
    H = np.zeros((n, n))
    H[1:, :-1] = np.eye(n - 1)               # ones on the subdiagonal
    H[:, -1] = -c[1:][::-1]                  # last column: -c_0, -c_1, ..., -c_{n-1}
    lam = ssd.hessenberg_eigenvalues(H)
    assert np.abs(lam.imag).max() < 1e-9
    assert np.sort(lam.real) == pytest.approx(np.sort(roots), abs=1e-9)


def test_complex_pairs_of_a_rotation_spectrum(ssd):
    rng = np.random.default_rng(8)
    blocks = [(0.5, 0.25), (-0.3, 1.0), (0.9, 0.05)]
    n = 2 * len(blocks) + 1
    B = np.zeros((n, n))
    for k, (a, b) in enumerate(blocks):
        B[2 * k:2 * k + 2, 2 * k:2 * k + 2] = [[a, b], [-b, a]]
    B[-1, -1] = 0.7
    Q = random_orthogonal(rng, n)
    H = reduce_to_hessenberg(Q @ B @ Q.T)
    lam = ssd.hessenberg_eigenvalues(H)
    ref = [complex(a, s * b) for a, b in blocks for s in (1, -1)] + [0.7]
    key = lambda z: (round(z.real, 9), round(z.imag, 9))
    assert np.array(sorted(lam, key=key)) == pytest.approx(np.array(sorted(ref, key=key)), abs=1e-12)


@pytest.mark.parametrize("spread", [1e-6, 1e-9, 0.0])
def test_clustered_spectrum_converges(ssd, spread):
    """Many eigenvalues in a tight cluster (as the D-N iteration matrix's high
    modes near 1/2), plus a few isolated ones, under an orthogonal similarity."""
    rng = np.random.default_rng(21)
    ev = np.concatenate([0.5 + spread * rng.normal(size=32), [0.9, -0.2, 0.05, 1.3]])
    n = ev.size
    Q = random_orthogonal(rng, n)
    H = reduce_to_hessenberg(Q @ np.diag(ev) @ Q.T)
    lam = ssd.hessenberg_eigenvalues(H)
    assert np.abs(lam.imag).max() < 1e-6
    assert np.sort(lam.real) == pytest.approx(np.sort(ev), abs=1e-7)
    assert backward_errors(H, lam).max() < 1e-11


def test_entries_below_the_subdiagonal_are_ignored(ssd):
    rng = np.random.default_rng(5)
    H = hessenberg(rng, 9)
    G = H + np.tril(rng.normal(size=(9, 9)), -2)
    assert np.array_equal(ssd.hessenberg_eigenvalues(H), ssd.hessenberg_eigenvalues(G))


def test_leading_block_of_an_arnoldi_matrix_with_leading_dimension(ssd):
    """ddm_spectrum returns H as (m+1) x m column-major: its k x k leading block
    is read in place with ldh = m + 1."""
    rng = np.random.default_rng(13)
    m, k = 10, 6
    Hfull = np.triu(rng.normal(size=(m + 1, m)), -1)
    buf = np.asfortranarray(Hfull)
    re = (ctypes.c_double * k)()
    im = (ctypes.c_double * k)()
    st = ssd.lib().ssd_hessenberg_eigenvalues(k, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), m + 1,
                                              re, im)
    assert st == 0
    got = np.array(re[:]) + 1j * np.array(im[:])
    assert np.array_equal(got, ssd.hessenberg_eigenvalues(Hfull[:k, :k]))


def test_invalid_arguments_and_input_left_unchanged(ssd):
    L = ssd.lib()
    P = ctypes.POINTER(ctypes.c_double)
    H = np.asfortranarray(np.triu(np.ones((4, 4)), -1))
    keep = H.copy()
    re = (ctypes.c_double * 4)()
    im = (ctypes.c_double * 4)()
    hp = H.ctypes.data_as(P)
    assert L.ssd_hessenberg_eigenvalues(0, hp, 4, re, im) == SSD_EINVAL
    assert L.ssd_hessenberg_eigenvalues(4, hp, 3, re, im) == SSD_EINVAL
    assert L.ssd_hessenberg_eigenvalues(4, None, 4, re, im) == SSD_EINVAL
    assert L.ssd_hessenberg_eigenvalues(4, hp, 4, None, im) == SSD_EINVAL
    assert L.ssd_hessenberg_eigenvalues(4, hp, 4, re, im) == 0
    assert np.array_equal(H, keep)
    H[2, 1] = np.nan
    assert L.ssd_hessenberg_eigenvalues(4, H.ctypes.data_as(P), 4, re, im) == SSD_EINVAL
    H[2, 1] = 1.0
    H[3, 0] = np.nan                          # below the subdiagonal: ignored
    assert L.ssd_hessenberg_eigenvalues(4, H.ctypes.data_as(P), 4, re, im) == 0
    with pytest.raises(ssd.SsdError):
        ssd.hessenberg_eigenvalues(np.full((3, 3), np.inf))
