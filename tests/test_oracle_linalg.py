"""Pins of the oracle's linear algebra: QR, symmetric eigen, two-sided Jacobi
SVD, entropy/truncation error (Eqs. 4-5), H_eff (Eq. 19), environments and
Lanczos.  Each check compares against something other than the oracle's own
formula: a library routine, a closed form, an invariant or an explicitly
built dense operator."""
import numpy as np
import pytest

import oracle as O
import synth

RNG = np.random.default_rng(1234)


def test_qr_factors():
    for m, n in [(7, 7), (12, 5), (40, 17)]:
        A = RNG.standard_normal((m, n))
        Q, R = O.qr(A)
        assert np.allclose(Q @ R, A, atol=1e-13)
        assert np.allclose(Q.T @ Q, np.eye(n), atol=1e-13)
        assert np.allclose(np.tril(R, -1), 0.0)


def test_sym_eig_matches_library():
    for n in [1, 2, 5, 20]:
        B = RNG.standard_normal((n, n))
        A = B + B.T
        w, Z = O.sym_eig(A)
        assert np.allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
        assert np.allclose(Z.T @ Z, np.eye(n), atol=1e-12)
        assert np.allclose(A @ Z, Z * w[None, :], atol=1e-11)


def test_svd_2x2_closed_form():
    # singular values of [[a, b], [c, d]]: (sqrt((a+d)^2+(c-b)^2) +- sqrt((a-d)^2+(b+c)^2)) / 2
    for _ in range(20):
        a, b, c, d = RNG.standard_normal(4)
        p = np.hypot(a + d, c - b)
        q = np.hypot(a - d, b + c)
        ref = np.array([(p + q) / 2, abs(p - q) / 2])
        U, s, Vt = O.svd(np.array([[a, b], [c, d]]))
        assert np.allclose(s, ref, rtol=1e-14, atol=1e-15)


def _sym3_eigvals(B):
    """Eigenvalues of a symmetric 3 x 3 matrix in closed form (Smith, CACM
    1961): with q = tr(B)/3, p^2 = |B - qI|_F^2 / 6 and r = det((B - qI)/p)/2,
    they are q + 2p cos(phi + 2 pi j/3), phi = acos(r)/3."""
    q = np.trace(B) / 3.0
    p1 = B[0, 1] ** 2 + B[0, 2] ** 2 + B[1, 2] ** 2
    p2 = (B[0, 0] - q) ** 2 + (B[1, 1] - q) ** 2 + (B[2, 2] - q) ** 2 + 2.0 * p1
    p = np.sqrt(p2 / 6.0)
    C = (B - q * np.eye(3)) / p
    detC = (C[0, 0] * (C[1, 1] * C[2, 2] - C[1, 2] * C[2, 1]) - C[0, 1] * (C[1, 0] * C[2, 2] - C[1, 2] * C[2, 0])
            + C[0, 2] * (C[1, 0] * C[2, 1] - C[1, 1] * C[2, 0]))
    phi = np.arccos(np.clip(detC / 2.0, -1.0, 1.0)) / 3.0
    e1 = q + 2.0 * p * np.cos(phi)
    e3 = q + 2.0 * p * np.cos(phi + 2.0 * np.pi / 3.0)
    return np.array([e1, 3.0 * q - e1 - e3, e3])


def test_svd_3x3_closed_form():
    """Squared singular values of a 3 x 3 matrix against the closed-form
    eigenvalues of A^T A, descending.  Forming A^T A and the formula carry an
    absolute error of a few eps |A|_F^2 per eigenvalue, so the comparison is
    on s^2 with that bar (the square root would amplify it for small s)."""
    eps = np.finfo(float).eps
    for _ in range(20):
        A = RNG.standard_normal((3, 3))
        ref = _sym3_eigvals(A.T @ A)
        U, s, Vt = O.svd(A)
        assert np.all(np.abs(s ** 2 - ref) <= 50 * eps * np.sum(A * A))
        assert np.all(np.diff(s) <= 0)
        assert np.allclose((U * s) @ Vt, A, atol=1e-14)


@pytest.mark.parametrize("kind", ["exp", "pow"])
@pytest.mark.parametrize("chi", [8, 32])
def test_svd_exact_spectrum(kind, chi):
    """A = U diag(s) V^T with Haar U, V and the prescribed spectra of the
    isolated-SVD workload: s is known exactly by construction."""
    n = 2 * chi
    s_ref = synth.spectrum(kind, n, chi)
    A = synth.svd_test_matrix(synth.workload_seed(1, chi), n, n, s_ref)
    U, s, Vt = O.svd(A)
    # Weyl: |s_k - s_ref_k| <= |dA|_2 with |dA| a few n*eps*|A| from forming A
    tol = 1e-10 * s_ref + 8 * n * np.finfo(float).eps * s_ref[0]
    assert np.all(np.abs(s - s_ref) <= tol)
    assert np.linalg.norm(U * s @ Vt - A) <= 1e-13 * np.linalg.norm(A)
    assert np.abs(U.T @ U - np.eye(n)).max() <= 1e-13
    assert np.abs(Vt @ Vt.T - np.eye(n)).max() <= 1e-13
    assert np.all(np.diff(s) <= 0)


@pytest.mark.parametrize("m,n", [(6, 9), (9, 6), (32, 16), (16, 40), (1, 5), (5, 1)])
def test_svd_rectangular_matches_library(m, n):
    A = RNG.standard_normal((m, n))
    U, s, Vt = O.svd(A)
    assert np.allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-12, atol=1e-13)
    assert np.allclose(U * s @ Vt, A, atol=1e-13)
    r = min(m, n)
    assert np.allclose(U.T @ U, np.eye(r), atol=1e-13)
    assert np.allclose(Vt @ Vt.T, np.eye(r), atol=1e-13)
    # sign convention: largest |entry| of every column of U is positive
    idx = np.argmax(np.abs(U), axis=0)
    assert np.all(U[idx, np.arange(r)] > 0)


def test_svd_rank_deficient():
    B = RNG.standard_normal((20, 3))
    A = B @ RNG.standard_normal((3, 15))
    U, s, Vt = O.svd(A)
    assert np.allclose(s[:3], np.linalg.svd(A, compute_uv=False)[:3], rtol=1e-12)
    assert np.all(s[3:] <= 1e-13 * s[0])
    assert np.allclose(U * s @ Vt, A, atol=1e-12)


def test_entropy_closed_forms():
    S, eps = O.entropy(np.array([1.0, 0.0, 0.0]))           # product state
    assert S == 0.0 and eps[1] == 0.0
    for chi in [2, 3, 7, 64, 1000]:                          # maximally entangled: S = ln chi
        S, _ = O.entropy(np.full(chi, 0.37))
        assert abs(S - np.log(chi)) <= 4e-15 * max(1.0, np.log(chi))
    S, _ = O.entropy(np.array([1.0, 1.0]) / np.sqrt(2))     # singlet: ln 2
    assert abs(S - np.log(2)) < 1e-15
    # scale invariance of Eq. (5) (p_k normalises the spectrum)
    s = np.sort(RNG.random(50))[::-1]
    assert abs(O.entropy(s)[0] - O.entropy(3.7 * s)[0]) < 1e-14


def test_truncation_error_is_eckart_young():
    """Eq. (4): eps_k = |theta - theta_k|_F / |theta|_F for the best rank-k approximation."""
    A = RNG.standard_normal((24, 18))
    U, s, Vt = np.linalg.svd(A, full_matrices=False)
    _, eps = O.entropy(s)
    for k in [1, 5, 17, 18]:
        Ak = (U[:, :k] * s[:k]) @ Vt[:k]
        assert abs(np.linalg.norm(A - Ak) / np.linalg.norm(A) - eps[k]) < 1e-14


def test_trunc_k_rules():
    s = np.array([0.8, 0.5, 0.3, 0.3, 0.3, 1e-12, 0.0])
    # chi limit, threshold on the normalised spectrum, multiplet guard
    assert O.trunc_k(s, 2, 1e-10) == 2
    assert O.trunc_k(s, 4, 1e-10, multiplet_guard=1) == 2      # would cut inside the 0.3 triplet
    assert O.trunc_k(s, 4, 1e-10, multiplet_guard=0) == 4
    assert O.trunc_k(s, 100, 1e-10) == 5                      # 1e-12 is below eps_trunc
    assert O.trunc_k(s, 100, 0.0) == 6                        # exact zero is beyond the rank
    assert O.trunc_k(np.array([0.0, 0.0]), 5, 1e-10) == 1     # never below 1


# ---------------------------------------------------------------------------
# H_eff and environments against a dense Hamiltonian built by Kronecker products
# ---------------------------------------------------------------------------
SZ = np.diag([0.5, -0.5]); SP = np.array([[0, 1.0], [0, 0]]); SM = SP.T.copy(); I2 = np.eye(2)


def kron_op(ops):
    out = np.ones((1, 1))
    for o in ops:
        out = np.kron(out, o)
    return out


def xxz_dense(N, J=1.0, Delta=1.0):
    H = np.zeros((2 ** N, 2 ** N))
    for i in range(N - 1):
        for a, b, c in [(SP, SM, 0.5 * J), (SM, SP, 0.5 * J), (SZ, SZ, J * Delta)]:
            ops = [I2] * N
            ops[i], ops[i + 1] = a, b
            H += c * kron_op(ops)
    return H


def random_canonical_mps(N, chi, rng):
    """Left-canonical sites 0..k-1 and right-canonical k+2..N-1 built with numpy QR."""
    dims = [min(chi, 2 ** i, 2 ** (N - i)) for i in range(N + 1)]
    A = [rng.standard_normal((dims[i], 2, dims[i + 1])) for i in range(N)]
    return dims, A


def test_heff_equals_projected_hamiltonian():
    rng = np.random.default_rng(7)
    N, chi, k = 6, 3, 2                       # bond between sites 2 and 3
    Delta, J = 0.7, 1.3
    dims, A = random_canonical_mps(N, chi, rng)
    W = O.mpo(O.MODEL_XXZ, N, J, Delta)
    # left-canonicalise sites < k, right-canonicalise sites > k+1 (numpy QR)
    for i in range(k):
        a, s, b = A[i].shape
        Q, R = np.linalg.qr(A[i].reshape(a * s, b))
        A[i] = Q.reshape(a, s, Q.shape[1])
    for i in range(N - 1, k + 1, -1):
        a, s, b = A[i].shape
        Q, R = np.linalg.qr(A[i].reshape(a, s * b).T)
        A[i] = Q.T.reshape(Q.shape[1], s, b)
    # dense isometries of the left and right blocks
    left = np.ones((1, 1))
    for i in range(k):
        a, s, b = A[i].shape
        left = np.einsum("xa,asb->xsb", left, A[i]).reshape(-1, b)
    right = np.ones((1, 1))
    for i in range(N - 1, k + 1, -1):
        a, s, b = A[i].shape
        right = np.einsum("asb,by->asy", A[i], right).reshape(a, -1)
    cl, cr = left.shape[1], right.shape[0]
    # environments through the oracle
    L = np.zeros((W.shape[1], 1, 1)); L[-1] = 1.0
    for i in range(k):
        L = O.env_left(L, W[i], A[i])
    R = np.zeros((W.shape[1], 1, 1)); R[0] = 1.0
    for i in range(N - 1, k + 1, -1):
        R = O.env_right(R, W[i], A[i])
    dim = cl * 4 * cr
    Heff = np.zeros((dim, dim))
    for c in range(dim):
        e = np.zeros(dim); e[c] = 1.0
        Heff[:, c] = O.heff_apply(L, W[k], W[k + 1], R, e.reshape(cl, 2, 2, cr)).ravel()
    # P maps theta[a][s1][s2][b] to the full state
    P = np.einsum("xa,ij,kl,by->xikyajlb", left, I2, I2, right).reshape(2 ** N, dim)
    Href = P.T @ xxz_dense(N, J, Delta) @ P
    assert np.allclose(Heff, Heff.T, atol=1e-13)
    assert np.allclose(Heff, Href, atol=1e-12)


def test_lanczos_against_dense_eigensolve():
    rng = np.random.default_rng(11)
    D, cl, cr = 5, 4, 3
    W = O.mpo(O.MODEL_XXZ, 4, 1.0, 1.0)
    # symmetric random environments (each w block symmetric keeps H_eff symmetric
    # only if paired; use environments from a real contraction instead)
    dims, A = random_canonical_mps(6, 4, rng)
    L = np.zeros((D, 1, 1)); L[-1] = 1.0
    for i in range(2):
        a, s, b = A[i].shape
        Q, _ = np.linalg.qr(A[i].reshape(a * s, b)); A[i] = Q.reshape(a, s, -1)
        L = O.env_left(L, W[0], A[i])
    R = np.zeros((D, 1, 1)); R[0] = 1.0
    for i in range(5, 3, -1):
        a, s, b = A[i].shape
        Q, _ = np.linalg.qr(A[i].reshape(a, s * b).T); A[i] = Q.T.reshape(-1, s, b)
        R = O.env_right(R, W[0], A[i])
    cl, cr = L.shape[1], R.shape[1]
    dim = cl * 4 * cr
    Heff = np.zeros((dim, dim))
    for c in range(dim):
        e = np.zeros(dim); e[c] = 1.0
        Heff[:, c] = O.heff_apply(L, W[2], W[3], R, e.reshape(cl, 2, 2, cr)).ravel()
    ev = np.linalg.eigvalsh(Heff)
    theta = rng.standard_normal((cl, 2, 2, cr))
    E, th, k, al, be = O.lanczos(L, W[2], W[3], R, theta, K=dim)
    assert abs(E - ev[0]) < 1e-10
    # tridiagonal eigenvalues vs library on T
    T = np.diag(al) + np.diag(be[:-1], 1) + np.diag(be[:-1], -1)
    assert abs(np.linalg.eigvalsh(T)[0] - E) < 1e-12
    # Ritz vector is an eigenvector of H_eff
    v = th.ravel()
    assert abs(np.linalg.norm(v) - 1) < 1e-12
    assert np.linalg.norm(Heff @ v - E * v) < 1e-7
    # with 20 steps on a larger space the Ritz value is an upper bound
    E20, *_ = O.lanczos(L, W[2], W[3], R, theta, K=3)
    assert E20 >= ev[0] - 1e-12


def _sturm_count(a, b, x):
    """Eigenvalues of the symmetric tridiagonal (a diagonal, b off-diagonal)
    below x: negative pivots of the LDL^T factorisation of T - x I."""
    cnt, q = 0, 1.0
    for i in range(len(a)):
        q = (a[i] - x) - (b[i - 1] ** 2 / q if i > 0 else 0.0)
        if q == 0.0:
            q = 1e-300
        cnt += q < 0.0
    return cnt


def _bisect_eig(a, b, k):
    """k-th smallest eigenvalue by bisection on Sturm counts (Gershgorin start)."""
    r = np.abs(np.r_[b, 0.0]) + np.abs(np.r_[0.0, b])
    lo, hi = float(np.min(a - r)), float(np.max(a + r))
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if mid in (lo, hi):
            break
        if _sturm_count(a, b, mid) > k:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def test_sym_eig_tridiagonal_against_sturm_bisection():
    """The eigensolver that also solves the Lanczos tridiagonal matrix, on
    T of the Lanczos sizes (K <= 20), against bisection on Sturm sequence
    counts written out here (Golub-Van Loan 8.4.1): every eigenvalue to 1e-13
    relative to |T|, including a glued pair of nearly equal ones."""
    rng = np.random.default_rng(11)
    for n in (1, 2, 7, 20):
        a = rng.standard_normal(n)
        b = rng.uniform(0.05, 1.0, n - 1)
        if n == 20:
            b[9] = 1e-9                                   # two nearly decoupled halves
        T = np.diag(a) + np.diag(b, 1) + np.diag(b, -1)
        w, _ = O.sym_eig(T)
        ref = np.array([_bisect_eig(a, b, k) for k in range(n)])
        assert np.max(np.abs(np.sort(w) - ref)) <= 1e-13 * max(1.0, np.max(np.abs(ref)))
