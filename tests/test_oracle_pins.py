"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own code (no GPU needed).

Each test builds its expectation another way: dense Kronecker operators,
numpy's FFT and SVD as library special cases, the block-circulant
characterisation of t-SVT (Section III-A, bcirc and Theorem 4.2), closed forms,
constructed t-SVDs and a dense brute-force ADMM iteration on 8x8x4 cubes.
"""
import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers --
def circ_diff(n):
    """Dense circulant forward difference: (C x)(i) = x(i+1) - x(i)."""
    C = -np.eye(n)
    for i in range(n):
        C[i, (i + 1) % n] += 1.0
    return C


def dense_D(shape):
    """D_1, D_2, D_3 as N x N matrices on Fortran-order vectors."""
    n1, n2, n3 = shape
    I1, I2, I3 = np.eye(n1), np.eye(n2), np.eye(n3)
    D1 = np.kron(I3, np.kron(I2, circ_diff(n1)))
    D2 = np.kron(I3, np.kron(circ_diff(n2), I1))
    D3 = np.kron(circ_diff(n3), np.kron(I2, I1))
    return D1, D2, D3


def vec(x):
    return np.asarray(x).reshape(-1, order="F")


def unvec(v, shape):
    return np.asarray(v).reshape(shape, order="F")


def svt_numpy(A, t):
    U, s, Vh = np.linalg.svd(A, full_matrices=False)
    return (U * np.maximum(s - t, 0.0)) @ Vh


def bcirc(A):
    """Block-circulant matrix of a cube (Section III-A): block (r, c) is the
    frontal slice (r - c) mod n3."""
    n1, n2, n3 = A.shape
    B = np.zeros((n1 * n3, n2 * n3), dtype=A.dtype)
    for r in range(n3):
        for c in range(n3):
            B[r * n1:(r + 1) * n1, c * n2:(c + 1) * n2] = A[:, :, (r - c) % n3]
    return B


def first_block_column(B, shape):
    n1, n2, n3 = shape
    return np.stack([B[k * n1:(k + 1) * n1, 0:n2] for k in range(n3)], axis=2)


def tsvt_bcirc(A, t):
    """t-SVT through the block-circulant matrix: SVT_t(bcirc(A)) is block
    circulant; its first block column is t-SVT_t(A)."""
    return first_block_column(svt_numpy(bcirc(A), t), A.shape).real


# ------------------------------------------------------- difference ops ---
@pytest.mark.parametrize("shape", [(5, 4, 3), (7, 1, 6), (8, 8, 4)])
def test_diff_matches_dense_kronecker(orc, shape):
    rng = np.random.default_rng(1)
    x = rng.standard_normal(shape)
    w = (0.7, 1.3, 0.4)
    g = orc.diff(x, w)
    for n, D in enumerate(dense_D(shape)):
        np.testing.assert_allclose(vec(g[n]), w[n] * (D @ vec(x)), atol=1e-13)


@pytest.mark.parametrize("shape", [(5, 4, 3), (6, 6, 5)])
def test_diff_adjoint_identity(orc, shape):
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape)
    g = rng.standard_normal((3,) + shape)
    w = (1.0, 0.5, 2.0)
    lhs = np.sum(orc.diff(x, w) * g)
    rhs = np.sum(x * orc.diff_adjoint(g, w))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    # and the adjoint equals the dense transpose
    D = dense_D(shape)
    ref = sum(w[n] * D[n].T @ vec(g[n]) for n in range(3))
    np.testing.assert_allclose(vec(orc.diff_adjoint(g, w)), ref, atol=1e-12)


def test_diff_rank_and_spectrum():
    """Circular D_n along a mode of length n has rank n-1 per fiber
    (Theorem 4.1's r(D) = np - 1) and D^T D has eigenvalues 4 sin^2(pi a/n)."""
    for n in (4, 5, 9):
        C = circ_diff(n)
        assert np.linalg.matrix_rank(C) == n - 1
        ev = np.sort(np.linalg.eigvalsh(C.T @ C))
        np.testing.assert_allclose(ev, np.sort(4 * np.sin(np.pi * np.arange(n) / n) ** 2), atol=1e-12)


def test_pz_closed_form(orc):
    shape = (6, 5, 4)
    w = (0.8, 1.1, 1.7)
    P = orc.pz(shape, w)
    a, b, c = np.meshgrid(*[np.arange(n) for n in shape], indexing="ij")
    ref = sum(w[n] ** 2 * 4 * np.sin(np.pi * idx / shape[n]) ** 2
              for n, idx in enumerate((a, b, c)))
    np.testing.assert_allclose(P, ref, atol=1e-12)
    # exactly one zero: the DC frequency (rank n - 1 of each D_n)
    assert np.sum(P < 1e-12) == 1 and P[0, 0, 0] < 1e-12


# ------------------------------------------------------------------ DFT ---
def test_dft_matches_fft(orc):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((6, 5, 7)) + 1j * rng.standard_normal((6, 5, 7))
    np.testing.assert_allclose(orc.dft3(a, -1), np.fft.fftn(a), atol=1e-11)
    np.testing.assert_allclose(orc.dft3(a, +1), np.fft.ifftn(a), atol=1e-12)
    for ax in range(3):
        np.testing.assert_allclose(orc.dft_axis(a, ax, -1), np.fft.fft(a, axis=ax), atol=1e-11)


def test_dft_roundtrip_parseval_symmetry(orc):
    rng = np.random.default_rng(4)
    x = rng.standard_normal((8, 3, 9))
    X = orc.dft3(x, -1)
    np.testing.assert_allclose(orc.dft3(X, +1).real, x, atol=1e-12)
    assert abs(np.sum(np.abs(X) ** 2) / x.size - np.sum(x ** 2)) < 1e-9
    # Hermitian symmetry of a real input's spectrum along mode 3
    Xk = orc.dft_axis(x, 2, -1)
    for k in range(1, 9):
        np.testing.assert_allclose(Xk[:, :, 9 - k], np.conj(Xk[:, :, k]), atol=1e-12)


# -------------------------------------------------------------- Z-solve ---
def test_zsolve_dense_brute_force(orc):
    shape = (8, 8, 4)
    rng = np.random.default_rng(5)
    T = rng.standard_normal(shape)
    w = (1.0, 0.6, 1.4)
    mu = 0.37
    D = dense_D(shape)
    A = mu * (np.eye(T.size) + sum(w[n] ** 2 * D[n].T @ D[n] for n in range(3)))
    ref = np.linalg.solve(A, vec(T))
    np.testing.assert_allclose(vec(orc.zsolve(T, mu, w)), ref, atol=1e-11)


def test_zsolve_stencil_residual(orc):
    shape = (12, 10, 7)
    rng = np.random.default_rng(6)
    T = rng.standard_normal(shape)
    w = (1.0, 1.0, 1.0)
    mu = 25.0
    Z = orc.zsolve(T, mu, w)
    back = mu * (Z + orc.diff_adjoint(orc.diff(Z, w), w))
    np.testing.assert_allclose(back, T, atol=1e-10)


# ------------------------------------------------------- soft threshold ---
def test_soft_threshold_prox(orc):
    v = np.array([-2.0, -0.3, -0.1, 0.0, 0.05, 0.1, 0.5, 3.0])
    d = 0.1
    x = orc.soft(v, d)
    np.testing.assert_allclose(x, np.sign(v) * np.maximum(np.abs(v) - d, 0), atol=0)
    # optimality: 0 in (x - v) + d * subdiff|x|
    for xi, vi in zip(x, v):
        if xi != 0:
            assert abs((xi - vi) + d * np.sign(xi)) < 1e-15
        else:
            assert abs(vi) <= d + 1e-15


# ------------------------------------------------------------------ SVT ---
@pytest.mark.parametrize("m,n", [(9, 6), (6, 9), (7, 7), (1, 5), (16, 16)])
def test_svt_matrix_vs_numpy(orc, m, n):
    rng = np.random.default_rng(m * 31 + n)
    A = rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))
    s = np.linalg.svd(A, compute_uv=False)
    np.testing.assert_allclose(orc.singular_values(A), s, atol=1e-12)
    for t in (0.0, 0.5 * s.min(), np.median(s), s.max() * 1.01):
        R, sw = orc.svt_matrix(A, t)
        assert sw > 0
        np.testing.assert_allclose(R, svt_numpy(A, t), atol=1e-11)


def test_svt_rank_deficient(orc):
    rng = np.random.default_rng(8)
    U = rng.standard_normal((20, 3)) + 1j * rng.standard_normal((20, 3))
    V = rng.standard_normal((3, 12)) + 1j * rng.standard_normal((3, 12))
    A = U @ V
    R, sw = orc.svt_matrix(A, 0.3)
    assert sw > 0
    np.testing.assert_allclose(R, svt_numpy(A, 0.3), atol=1e-10)


@pytest.mark.parametrize("shape", [(8, 8, 4), (6, 5, 4), (4, 7, 5)])
def test_tsvt_equals_bcirc_svt(orc, shape):
    rng = np.random.default_rng(9)
    A = rng.standard_normal(shape)
    sig = np.linalg.svd(bcirc(A), compute_uv=False)
    for t in (0.0, np.percentile(sig, 30), np.percentile(sig, 80)):
        out, sw = orc.tsvt(A, t)
        assert sw > 0
        np.testing.assert_allclose(out, tsvt_bcirc(A, t), atol=1e-10)


def test_tsvt_exact_recovery_from_built_tsvd(orc):
    """A = U * S * V^T built from per-Fourier-slice unitary factors and known
    singular values (conjugate-symmetric in k, so A is real); then
    t-SVT_t(A) = U * (S - t)_+ * V^T slice by slice."""
    n1, n2, n3 = 9, 7, 6
    rng = np.random.default_rng(10)
    h = n3 // 2 + 1
    Ah = np.zeros((n1, n2, n3), complex)
    Rh = np.zeros((n1, n2, n3), complex)
    t = 1.5
    for k in range(h):
        real_slice = (k == 0) or (2 * k == n3)
        M1 = rng.standard_normal((n1, n1)) + (0 if real_slice else 1j) * rng.standard_normal((n1, n1))
        M2 = rng.standard_normal((n2, n2)) + (0 if real_slice else 1j) * rng.standard_normal((n2, n2))
        U = np.linalg.qr(M1)[0]
        V = np.linalg.qr(M2)[0]
        s = np.sort(rng.uniform(0.2, 4.0, min(n1, n2)))[::-1]
        Sm = np.zeros((n1, n2))
        Sm[np.arange(len(s)), np.arange(len(s))] = s
        St = np.zeros((n1, n2))
        St[np.arange(len(s)), np.arange(len(s))] = np.maximum(s - t, 0)
        Ah[:, :, k] = U @ Sm @ V.conj().T
        Rh[:, :, k] = U @ St @ V.conj().T
        if 0 < k and 2 * k != n3:
            Ah[:, :, n3 - k] = np.conj(Ah[:, :, k])
            Rh[:, :, n3 - k] = np.conj(Rh[:, :, k])
    A = np.fft.ifft(Ah, axis=2)
    R = np.fft.ifft(Rh, axis=2)
    assert np.max(np.abs(A.imag)) < 1e-12
    out, sw = orc.tsvt(A.real, t)
    assert sw > 0
    np.testing.assert_allclose(out, R.real, atol=1e-11)
    # tensor nuclear norm = sum_i S(i, i, 1) = (1/n3) sum_k ||A_k||_* (Theorem 4.2)
    tnn = sum(orc.singular_values(Ah[:, :, k]).sum() for k in range(n3)) / n3
    assert abs(tnn - np.sum(np.linalg.svd(bcirc(A.real), compute_uv=False)) / n3) < 1e-9


def test_tsvt_limits(orc):
    rng = np.random.default_rng(11)
    A = rng.standard_normal((6, 5, 4))
    out, _ = orc.tsvt(A, 0.0)
    np.testing.assert_allclose(out, A, atol=1e-12)
    big = np.linalg.svd(bcirc(A), compute_uv=False).max() * 1.001
    out, _ = orc.tsvt(A, big)
    np.testing.assert_allclose(out, 0.0, atol=1e-12)


# ----------------------------------------------------------------- ADMM ---
def brute_force_iteration(st, shape, p, mu, fstep=None):
    """One ADMM iteration of Section III-C written with dense matrices,
    numpy's dense solve and the block-circulant t-SVT; state is a dict.
    fstep(v, mu), when given, replaces the F-update's soft threshold of the
    stacked 3N-vector v."""
    tau, alpha, lam, w = p["tau"], p["alpha"], p["lam"], p["w"]
    D = dense_D(shape)
    Dw = np.vstack([w[n] * D[n] for n in range(3)])
    N = int(np.prod(shape))
    Y, S, Z, G1, G2 = (vec(st[k]) for k in ("Y", "S", "Z", "G1", "G2"))
    F = np.concatenate([vec(st["F"][n]) for n in range(3)])
    E = np.concatenate([vec(st["E"][n]) for n in range(3)])
    G3 = np.concatenate([vec(st["G3"][n]) for n in range(3)])
    G4 = np.concatenate([vec(st["G4"][n]) for n in range(3)])
    L = 0.5 * (Y - S + Z + (G1 - G2) / mu)
    T = mu * L + mu * Dw.T @ F + G2 - Dw.T @ G3
    Z = np.linalg.solve(mu * (np.eye(N) + Dw.T @ Dw), T)
    DZ = Dw @ Z
    v = 0.5 * ((DZ + G3 / mu) + (E + G4 / mu))
    F = np.sign(v) * np.maximum(np.abs(v) - tau / mu, 0) if fstep is None else fstep(v, mu)
    E = np.concatenate([vec(tsvt_bcirc(unvec(F[n * N:(n + 1) * N] - G4[n * N:(n + 1) * N] / mu,
                                             shape), alpha / mu)) for n in range(3)])
    u = Y - L + G1 / mu
    S = np.sign(u) * np.maximum(np.abs(u) - lam / mu, 0)
    G1 = G1 + mu * (Y - L - S)
    G2 = G2 + mu * (L - Z)
    G3 = G3 + mu * (DZ - F)
    G4 = G4 + mu * (E - F)
    split = lambda a: np.stack([unvec(a[n * N:(n + 1) * N], shape) for n in range(3)])
    return {"Y": st["Y"], "L": unvec(L, shape), "Z": unvec(Z, shape), "S": unvec(S, shape),
            "G1": unvec(G1, shape), "G2": unvec(G2, shape), "F": split(F), "E": split(E),
            "G3": split(G3), "G4": split(G4)}


def test_admm_iterations_brute_force(orc):
    shape = (8, 8, 4)
    rng = np.random.default_rng(12)
    Y = np.clip(rng.uniform(0, 1, shape) + 0.1 * rng.standard_normal(shape), -0.2, 1.2)
    P = orc.Params(tau=0.01, alpha=0.3, lam=0.05, w=(1.0, 0.8, 1.2), mu0=0.5, rho=1.7)
    st = orc.State(Y, P)
    bf = {"Y": Y, "L": Y.copy(), "Z": Y.copy(), "S": np.zeros(shape), "G1": np.zeros(shape),
          "G2": np.zeros(shape), "F": np.zeros((3,) + shape), "E": np.zeros((3,) + shape),
          "G3": np.zeros((3,) + shape), "G4": np.zeros((3,) + shape)}
    pd = {"tau": P.tau, "alpha": P.alpha, "lam": P.lam, "w": P.w}
    mu = P.mu0
    for _ in range(3):
        bf = brute_force_iteration(bf, shape, pd, mu)
        mu = min(P.rho * mu, P.mu_max)
    st.iterate(3)
    assert abs(st.mu - mu) < 1e-15
    for name in ("L", "Z", "S", "G1", "G2"):
        np.testing.assert_allclose(st.get(name), bf[name], atol=1e-9, err_msg=name)
    for name in ("F", "E", "G3", "G4"):
        for n in range(3):
            np.testing.assert_allclose(st.get(name, n), bf[name][n], atol=1e-9, err_msg=name)


# ------------------------------------------------- isotropic LRSTV (F) ---
def _nelder_mead_min(f, x0):
    from scipy.optimize import minimize
    best = None
    for start in (x0, np.zeros_like(x0), 0.5 * x0):
        r = minimize(f, start, method="Nelder-Mead",
                     options={"xatol": 1e-13, "fatol": 1e-16, "maxiter": 20000, "maxfev": 40000})
        if best is None or r.fun < best.fun:
            best = r
    return best.x


def test_group_soft_is_the_prox_of_the_two_norm(orc):
    """x = argmin 1/2 |x - v|^2 + d |x|_2, found by a derivative-free minimiser;
    in one dimension it is the scalar soft threshold; it commutes with
    rotations; inside the ball |v| <= d it is zero."""
    rng = np.random.default_rng(31)
    for m in (1, 2, 3, 4):
        for _ in range(4):
            v = rng.standard_normal(m)
            d = float(rng.uniform(0.1, 1.5))
            x = orc.group_soft(v, d)[0]
            ref = _nelder_mead_min(lambda y: 0.5 * np.sum((y - v) ** 2) + d * np.linalg.norm(y), v)
            assert np.max(np.abs(x - ref)) < 1e-6, (m, v, d)
            if m == 1:
                assert abs(x[0] - orc.soft(v, d)[0]) < 1e-15
    v = rng.standard_normal(3)
    Q, _ = np.linalg.qr(rng.standard_normal((3, 3)))
    np.testing.assert_allclose(orc.group_soft(Q @ v, 0.4)[0], Q @ orc.group_soft(v, 0.4)[0],
                               atol=1e-14)
    inside = 0.3 * v / np.linalg.norm(v)
    assert np.all(orc.group_soft(inside, 0.3 + 1e-12)[0] == 0.0)


@pytest.mark.parametrize("exact", [False, True])
def test_iso_admm_iterations_brute_force(orc, exact):
    """Isotropic LRSTV (eq. CRSSTV_iso, per-voxel 2-norm): the oracle's F-update
    against the F-subproblem kappa sum_v |F_v|_2 + mu/2 (|a - F|^2 + |b - F|^2)
    minimised voxel by voxel with a derivative-free minimiser (kappa = tau for
    the exact minimiser's reading, 2 tau for the printed tau/mu threshold)."""
    shape = (6, 5, 4)
    N = int(np.prod(shape))
    rng = np.random.default_rng(14)
    Y = np.clip(rng.uniform(0, 1, shape) + 0.1 * rng.standard_normal(shape), -0.2, 1.2)
    P = orc.Params(tau=0.05, alpha=0.3, lam=0.05, w=(1.0, 0.8, 1.2), mu0=0.5, rho=1.7)
    flags = orc.FLAG_ISO_TV | (orc.FLAG_F_THRESH_EXACT if exact else 0)
    st = orc.State(Y, P, flags=flags)
    kappa = P.tau if exact else 2 * P.tau

    def fstep(v, mu):
        # v = (a + b)/2 and |a-F|^2 + |b-F|^2 = 2 |F - v|^2 + const
        V = v.reshape(3, N).T
        out = np.empty_like(V)
        for k in range(N):
            out[k] = _nelder_mead_min(lambda y: kappa * np.linalg.norm(y) + mu * np.sum((y - V[k]) ** 2),
                                      V[k])
        return out.T.reshape(-1)

    bf = {"Y": Y, "L": Y.copy(), "Z": Y.copy(), "S": np.zeros(shape), "G1": np.zeros(shape),
          "G2": np.zeros(shape), "F": np.zeros((3,) + shape), "E": np.zeros((3,) + shape),
          "G3": np.zeros((3,) + shape), "G4": np.zeros((3,) + shape)}
    pd = {"tau": P.tau, "alpha": P.alpha, "lam": P.lam, "w": P.w}
    mu = P.mu0
    for _ in range(2):
        bf = brute_force_iteration(bf, shape, pd, mu, fstep)
        mu = min(P.rho * mu, P.mu_max)
    st.iterate(2)
    for name in ("L", "Z", "S", "G1", "G2"):
        np.testing.assert_allclose(st.get(name), bf[name], atol=1e-6, err_msg=name)
    for name in ("F", "E", "G3", "G4"):
        for n in range(3):
            np.testing.assert_allclose(st.get(name, n), bf[name][n], atol=1e-6, err_msg=name)
    # the group threshold zeroes whole voxels: F_1, F_2, F_3 vanish together
    F = np.stack([st.get("F", n) for n in range(3)])
    zero = np.all(F == 0.0, axis=0)
    assert zero.any() and not zero.all()


def test_iso_residuals_vanish_and_differ_from_anisotropic(orc):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(16, 16, 8, 3, 6, (0.1, 0.1), 0.1), 3)
    iso = orc.State(noisy, orc.Params(n1=16, n2=16), flags=orc.FLAG_ISO_TV)
    res, _ = iso.iterate(60)
    assert res[-1].max() < 1e-5
    ani = orc.State(noisy, orc.Params(n1=16, n2=16))
    ani.iterate(60)
    assert np.max(np.abs(iso.X - ani.X)) > 1e-4


def test_admm_residuals_vanish(orc):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(16, 16, 8, 3, 6, (0.1, 0.1), 0.1), 3)
    st = orc.State(noisy, orc.Params(n1=16, n2=16))
    res, sw = st.iterate(60)
    assert sw > 0
    assert res[-1].max() < 1e-5
    assert res[-1].max() < 1e-2 * res[5].max()
    # the extra constraint E = F is met as well (with the Gamma4 update)
    ef = max(np.max(np.abs(st.get("E", n) - st.get("F", n))) for n in range(3))
    assert ef < 1e-5


def test_alpha_zero_is_sstv(orc):
    """alpha = 0 switches the low-rank term off (LRSTV -> SSTV, Section III-A):
    the E-update is then E = F - Gamma4/mu exactly."""
    rng = np.random.default_rng(13)
    Y = rng.uniform(0, 1, (6, 6, 5))
    st = orc.State(Y, orc.Params(alpha=0.0, n1=6, n2=6))
    st.iterate(2)
    st.step_l(); st.step_z(); st.step_f(); st.step_e()
    for n in range(3):
        np.testing.assert_allclose(st.get("E", n), st.get("F", n) - st.get("G4", n) / st.mu,
                                   atol=1e-12)


def test_noise_free_constant_cube_is_fixed_point(orc):
    """A constant cube has zero gradients: F = E = 0 and L = Y stay fixed."""
    Y = np.full((6, 5, 4), 0.37)
    st = orc.State(Y, orc.Params(n1=6, n2=5))
    st.iterate(5)
    np.testing.assert_allclose(st.X, Y, atol=1e-12)


# ------------------------------------------------------------ generator ---
def test_generator_noisy_psnr_matches_paper():
    """Gaussian noise of 'variance' G gives the paper's noisy MPSNR (Tables I
    and II, cases 1 and 2), which fixes G as a standard deviation on [0, 1]
    data; the Pavia entries are checked at the Pavia shape, 200 x 200 x 80."""
    from synthetic import Recipe, make_cube, mpsnr
    gold = json.load(open(os.path.join(GOLDEN, "paper_noisy_psnr.json")))
    for key, sigma, shape in (("case1_gaussian_0.1", 0.1, (64, 64, 32)),
                              ("case2_gaussian_0.2", 0.2, (64, 64, 32)),
                              ("pavia_case1_gaussian_0.1", 0.1, (200, 200, 80)),
                              ("pavia_case2_gaussian_0.2", 0.2, (200, 200, 80))):
        clean, noisy = make_cube(Recipe(*shape, 4, 12, (sigma, sigma), 0.0), 7)
        assert abs(mpsnr(noisy, clean) - gold[key]["noisy_mpsnr_db"]) < 0.05, key


def test_generator_is_deterministic_and_in_range():
    from synthetic import RECIPES, make_cube
    c1, y1 = make_cube(RECIPES["c1"], 1)
    c2, y2 = make_cube(RECIPES["c1"], 1)
    assert np.array_equal(y1, y2)
    assert c1.min() >= 0 and c1.max() <= 1 + 1e-12
    _, y3 = make_cube(RECIPES["c1"], 2)
    assert not np.array_equal(y1, y3)
