"""Pins of the FP64 Tucker/HOOI L-update (oracle/tucker.py) against facts
that do not depend on its code: the Kronecker form of the projection, exact
recovery of a tensor of the stated multilinear rank, the Eckart-Young best
low-rank matrix in the one-band case, the monotone fit of alternating
least squares, and the full-rank case, which is the plain L-update."""
import numpy as np
import pytest

from oracle import tucker as tk


def _orth(rng, n, r):
    q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    return q[:, :r]


def vec(x):
    return np.asarray(x).reshape(-1, order="F")


def test_projection_is_the_kronecker_projector():
    rng = np.random.default_rng(1)
    shape, ranks = (5, 4, 3), (3, 2, 2)
    X = rng.standard_normal(shape)
    U = [_orth(rng, shape[n], ranks[n]) for n in range(3)]
    P = [u @ u.T for u in U]
    # vec in Fortran order: mode 1 fastest, so the operator is P3 (x) P2 (x) P1
    K = np.kron(P[2], np.kron(P[1], P[0]))
    assert np.max(np.abs(vec(tk.project(X, U)) - K @ vec(X))) < 1e-12


def test_exact_multilinear_rank_is_recovered():
    rng = np.random.default_rng(2)
    shape, ranks = (9, 8, 7), (4, 3, 2)
    C = rng.standard_normal(ranks)
    Q = [_orth(rng, shape[n], ranks[n]) for n in range(3)]
    X = tk.project(C, [np.eye(r) for r in ranks])  # the core itself
    for n in range(3):
        X = tk.mode_product(X, Q[n], n)
    L, U = tk.tucker_l_update(X, None, ranks)
    assert np.max(np.abs(L - X)) < 1e-11
    for n in range(3):
        assert np.max(np.abs(U[n].T @ U[n] - np.eye(ranks[n]))) < 1e-12


def test_full_ranks_are_the_identity():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((6, 5, 4))
    L, _ = tk.tucker_l_update(X, None, X.shape)
    assert np.max(np.abs(L - X)) < 1e-12


def test_one_band_case_converges_to_eckart_young():
    """With n3 = r3 = 1 the Tucker model is a rank-r matrix and HOOI is an
    alternating subspace iteration: it reaches the best rank-r approximation."""
    rng = np.random.default_rng(4)
    n1, n2, r = 12, 10, 3
    A = (_orth(rng, n1, n2) * np.linspace(10, 1, n2)) @ _orth(rng, n2, n2).T  # sigma 10 .. 1
    X = A[:, :, None]
    U = None
    for _ in range(60):
        L, U = tk.tucker_l_update(X, U, (r, r, 1))
    u, s, vt = np.linalg.svd(A)
    best = (u[:, :r] * s[:r]) @ vt[:r]
    assert np.max(np.abs(L[:, :, 0] - best)) < 1e-9


def test_hooi_fit_never_decreases_and_beats_hosvd():
    rng = np.random.default_rng(5)
    shape, ranks = (10, 9, 8), (5, 4, 3)
    X = rng.standard_normal(shape)
    U = tk.hosvd(X, ranks)
    fits = [np.linalg.norm(tk.project(X, U))]
    for _ in range(8):
        U = tk.hooi_sweep(X, U, ranks)
        fits.append(np.linalg.norm(tk.project(X, U)))
    assert all(b >= a - 1e-12 for a, b in zip(fits, fits[1:]))
    assert fits[-1] > fits[0]


def test_full_rank_tdlrstv_equals_the_plain_iteration(orc):
    from synthetic import Recipe, make_cube
    _, Y = make_cube(Recipe(8, 7, 5, 3, 5, (0.1, 0.1), 0.1), 6)
    p = orc.Params(n1=8, n2=7)
    plain = orc.State(Y, p)
    plain.iterate(4)
    tuck = tk.TuckerState(orc, Y, p, (8, 7, 5))
    tuck.iterate(4)
    for name in ("L", "Z", "S", "G1", "G2"):
        assert np.max(np.abs(plain.get(name) - tuck.st.get(name))) < 1e-10, name
    assert abs(plain.mu - tuck.st.mu) < 1e-15


# -------------------------------------------------- planted mistakes ---
def test_pins_catch_planted_mistakes(monkeypatch):
    """Plausible mistakes in the HOOI reference each fail a pin above: the
    smallest eigenvectors instead of the largest, a mode left out of the
    projection, and a sweep that ignores the other modes' factors."""
    def smallest(G, r):
        w, V = np.linalg.eigh(G)
        return V[:, :r]

    with monkeypatch.context() as m:
        m.setattr(tk, "leading_eigvecs", smallest)
        with pytest.raises(AssertionError):
            test_exact_multilinear_rank_is_recovered()

    def project_two_modes(X, U):
        C = X
        for n in range(2):
            C = tk.mode_product(C, U[n].T, n)
        for n in range(2):
            C = tk.mode_product(C, U[n], n)
        return C

    with monkeypatch.context() as m:
        m.setattr(tk, "project", project_two_modes)
        with pytest.raises(AssertionError):
            test_projection_is_the_kronecker_projector()

    def sweep_ignoring_other_factors(X, U, ranks):
        # each factor from the Gram of X itself: the HOSVD again, no HOOI
        return tk.hosvd(X, ranks)

    with monkeypatch.context() as m:
        m.setattr(tk, "hooi_sweep", sweep_ignoring_other_factors)
        with pytest.raises(AssertionError):
            test_hooi_fit_never_decreases_and_beats_hosvd()
