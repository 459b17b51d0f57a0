"""GPU parity of the full TDLRSTV L-update (lrstv_plan_set_tucker): the Tucker
projection by one HOOI sweep per ADMM iteration, against the FP64 reference
(oracle/tucker.py, whose other steps are the C oracle's).

Tolerance.  A factor's error is about the Gram matrix's rounding over the
eigenvalue gap at the rank cut.  On cubes of the stated multilinear rank plus
Gaussian noise, cut at that rank, the gap is 0.4-4% of the largest eigenvalue
and whole iterations are held to the 1e-4 max-abs bound of the plain path.
With the paper's ranks (r1 = 0.8 n1, r2 = 0.8 n2) on the mixed-noise recipe
the cut falls inside the noise's eigenvalue bulk (gaps of 1e-6 to 1e-4 of the
largest eigenvalue): FP32 and FP64 then keep different, equally valid
subspaces there, so that case checks the validity of every factor the GPU
computes against an FP64 replay of its own HOOI sweep (orthonormality, the
Rayleigh quotient, the well-separated eigenvectors, the projection and the
HOOI objective), and the final denoising quality to 0.01 dB.
"""
import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def _noisy(shape, seed, endmembers=4):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(*shape, endmembers, 12, (0.1, 0.1), 0.1), seed)
    return f32(clean), f32(noisy)


def _run(L, shape, ranks, iters, Y, flags=0):
    p = L.Params.make(shape[0], shape[1], max_iter=iters, flags=flags)
    with L.Plan(*shape, p) as pl:
        if ranks is not None:
            pl.set_tucker(ranks)
        X, S, st = pl.run(dev(Y), stats=True)
        assert st.jacobi_unconverged == 0 and st.gemm_errors == 0
        return host(X, shape), host(S, shape)


def _low_rank(shape, r, seed, noise=0.02):
    """A cube of multilinear rank (r, r, r) (a constant component and r - 1
    seeded directions per mode, superdiagonal core) plus Gaussian noise."""
    rng = np.random.default_rng(seed)
    Q = []
    for n in shape:
        M = rng.standard_normal((n, r))
        M[:, 0] = 1.0
        q = np.linalg.qr(M)[0]
        Q.append(q * np.sign(q[0, 0]))
    s = np.sqrt(np.prod(shape)) * np.concatenate([[0.5], np.linspace(0.2, 0.1, r - 1)])
    clean = sum(s[i] * np.einsum("a,b,c->abc", Q[0][:, i], Q[1][:, i], Q[2][:, i])
                for i in range(r))
    return f32(clean), f32(clean + noise * rng.standard_normal(shape))


@pytest.mark.parametrize("shape,r,iters", [((24, 20, 9), 3, 8), ((20, 24, 8), 3, 8),
                                           ((64, 64, 31), 4, 15)])
def test_tucker_run_matches_oracle(L, orc, shape, r, iters):
    from oracle import tucker as tk
    ranks = (r, r, r)
    clean, Y = _low_rank(shape, r, 21)
    X, S = _run(L, shape, ranks, iters, Y)
    ref = tk.TuckerState(orc, Y, orc.Params(n1=shape[0], n2=shape[1]), ranks)
    ref.iterate(iters)
    print(shape, ranks, "max-abs", maxabs(X, ref.X), "S", maxabs(S, ref.st.get("S")))
    assert maxabs(X, ref.X) <= 1e-4
    assert maxabs(S, ref.st.get("S")) <= 1e-4


def _gram_chain(X, U, mode):
    """The mode-n Gram matrix of one HOOI step: X multiplied by the other
    factors' transposes, unfolded along `mode`, times its transpose."""
    from oracle import tucker as tk
    Z = X
    for m in range(3):
        if m != mode:
            Z = tk.mode_product(Z, U[m].T, m)
    Zn = tk.unfold(Z, mode)
    return Zn @ Zn.T


def test_tucker_paper_ranks_validity(L, orc):
    """The paper's ranks (r1 = 0.8 n1, r2 = 0.8 n2, r3 = 6; Section IV-D) on
    the mixed-noise recipe, 64x64x31, 15 iterations.  The cut falls inside the
    noise's eigenvalue bulk (gaps of 1e-6 to 1e-4 of the largest eigenvalue),
    where the FP32 and FP64 eigen-solves may keep different, equally valid
    subspaces, so the GPU's own HOOI sweep is replayed in FP64 every
    iteration (target X from the GPU's state, the GPU's factors for the
    modes already updated) and its result is checked for validity:
     - each factor has orthonormal columns (to 1e-5);
     - its Rayleigh quotient trace(U^T G U) on the FP64 Gram matrix G of its
       HOOI step reaches the sum of G's r leading eigenvalues to 1e-5 of that
       sum: with G's FP32 rounding ||E|| <= eta, the eigenvectors of G + E lose
       at most 2 r eta, and eta is ~1e-7 of the trace here;
     - every leading eigenvector of G whose gap to the cut, lambda_i -
       lambda_{r+1}, exceeds 1e-3 lambda_1 lies in span(U) up to the
       Davis-Kahan bound 8 n eps32 lambda_1 / gap (FP32 Gram rounding of about
       n eps32 lambda_1 over that gap);
     - the projection L = X x1 U1 U1^T x2 U2 U2^T x3 U3 U3^T equals the FP64
       projection of X with the GPU's factors to 1e-5;
     - the HOOI objective ||X x1 U1^T x2 U2^T x3 U3^T||^2 is within 1e-5 of
       the FP64 sweep's from the same start.
    After the 15 iterations the MPSNR is that of the FP64 reference to 0.01 dB."""
    import torch
    from oracle import tucker as tk
    from synthetic import mpsnr
    shape, iters = (64, 64, 31), 15
    ranks = (51, 51, 6)
    eps32 = 2.0 ** -24
    clean, Y = _noisy(shape, 21)
    p = L.Params.make(64, 64, max_iter=iters)
    U_prev = None
    with L.Plan(*shape, p) as pl:
        pl.set_tucker(ranks)
        pl.init(dev(Y))
        for k in range(iters):
            g = {n: host(pl.get(n), shape) for n in ("Y", "S", "Z", "G1", "G2")}
            mu = pl.mu[0]
            X = 0.5 * (g["Y"] - g["S"] + g["Z"] + (g["G1"] - g["G2"]) / mu)
            pl.iterate(1)
            torch.cuda.synchronize()
            U = [pl.tucker_factor(n, ranks[n]).cpu().numpy().astype(np.float64) for n in range(3)]
            start = tk.hosvd(X, ranks) if U_prev is None else U_prev
            chain = list(start)
            for n in range(3):
                assert np.abs(U[n].T @ U[n] - np.eye(ranks[n])).max() <= 1e-5, (k, n)
                G = _gram_chain(X, chain, n)
                lam, V = np.linalg.eigh(G)
                lam, V = lam[::-1], V[:, ::-1]
                r = ranks[n]
                top = lam[:r].sum()
                rq = np.trace(U[n].T @ G @ U[n])
                assert top - rq <= 1e-5 * top, (k, n, top, rq)
                if r < len(lam):
                    for i in range(r):
                        gap = lam[i] - lam[r]
                        if gap > 1e-3 * lam[0]:
                            v = V[:, i]
                            off = np.linalg.norm(v - U[n] @ (U[n].T @ v))
                            assert off <= 8 * G.shape[0] * eps32 * lam[0] / gap, (k, n, i, off)
                chain[n] = U[n]  # the next mode's step uses this mode's new factor
            Lg = host(pl.get("L"), shape)
            assert maxabs(Lg, tk.project(X, U)) <= 1e-5, k
            ref = tk.hooi_sweep(X, start, ranks)
            obj = lambda W: float(np.sum(tk.project(X, W) ** 2))
            assert abs(obj(U) - obj(ref)) <= 1e-5 * obj(ref), k
            U_prev = U
        Xg = host(pl.get("L"), shape)
    refst = tk.TuckerState(orc, Y, orc.Params(n1=64, n2=64), ranks)
    refst.iterate(iters)
    d = mpsnr(Xg, clean) - mpsnr(refst.X, clean)
    print("MPSNR GPU / FP64:", mpsnr(Xg, clean), mpsnr(refst.X, clean), "max-abs",
          maxabs(Xg, refst.X))
    assert abs(d) <= 0.01


def test_full_ranks_equal_the_plain_plan(L):
    shape = (24, 20, 9)
    _, Y = _noisy(shape, 22)
    X0, _ = _run(L, shape, None, 6, Y)
    X1, _ = _run(L, shape, shape, 6, Y)
    assert maxabs(X0, X1) <= 1e-5


def test_tucker_warm_start_and_graph(L, orc):
    """The warm-started Jacobi of the E-step and graph replay combine with the
    Tucker L-update (the factors restart from the HOSVD at every run)."""
    import torch
    from oracle import tucker as tk
    shape, ranks, iters = (24, 20, 9), (3, 3, 3), 8
    _, Y = _low_rank(shape, 3, 23)
    p = L.Params.make(24, 20, max_iter=iters, flags=L.FLAG_WARM_START | L.FLAG_GRAPH)
    with L.Plan(*shape, p) as pl:
        pl.set_tucker(ranks)
        X1, _ = pl.run(dev(Y))
        X2, _ = pl.run(dev(Y))
        torch.cuda.synchronize()
        assert torch.equal(X1, X2)
        X = host(X1, shape)
    ref = tk.TuckerState(orc, Y, orc.Params(n1=24, n2=20), ranks)
    ref.iterate(iters)
    assert maxabs(X, ref.X) <= 1e-4


def test_tucker_argument_checks(L):
    p = L.Params.make(8, 8)
    with L.Plan(8, 8, 4, p) as pl:
        for bad in ((0, 4, 2), (9, 4, 2), (4, 4, 5), (-1, 4, 2)):
            with pytest.raises(L.LrstvError, match="status 1"):
                pl.set_tucker(bad)
        pl.set_tucker((6, 6, 2))
        pl.set_tucker(None)
        pl.set_tucker((0, 0, 0))
    with L.Plan(8, 8, 600, L.Params.make(8, 8)) as pl:
        with pytest.raises(L.LrstvError, match="status 2"):
            pl.set_tucker((6, 6, 2))


def test_tucker_with_the_isotropic_variant(L, orc):
    """Both NEXT-4 parts together: the Tucker L-update and the isotropic
    F-update, against the FP64 reference run with the oracle's isotropic flag."""
    from oracle import tucker as tk
    shape, ranks, iters = (24, 20, 9), (3, 3, 3), 8
    _, Y = _low_rank(shape, 3, 31)
    X, S = _run(L, shape, ranks, iters, Y, flags=L.FLAG_ISO_TV)
    ref = tk.TuckerState(orc, Y, orc.Params(n1=24, n2=20), ranks, flags=orc.FLAG_ISO_TV)
    ref.iterate(iters)
    assert maxabs(X, ref.X) <= 1e-4
    assert maxabs(S, ref.st.get("S")) <= 1e-4


def test_tucker_inside_a_batch_equals_the_plan(L):
    """A batch whose second cube has the Tucker L-update (set through
    lrstv_batch_plan) gives, for every cube, the standalone plan's bits."""
    import torch
    shapes = [(24, 20, 9), (20, 24, 8), (32, 32, 6)]
    Ys = [dev(_low_rank(s, 3, 40 + i)[1]) for i, s in enumerate(shapes)]
    p = L.Params.make(24, 20, max_iter=6)
    with L.Batch(shapes, p) as b:
        b.plan(1).set_tucker((3, 3, 3))
        Xs, _ = b.run(Ys)
        torch.cuda.synchronize()
        got = [x.cpu() for x in Xs]
    p1 = L.Params.make(24, 20, max_iter=6, flags=L.FLAG_JACOBI_PER_SLICE)  # a batch's order
    for i, sh in enumerate(shapes):
        with L.Plan(*sh, p1) as pl:
            if i == 1:
                pl.set_tucker((3, 3, 3))
            X, _ = pl.run(Ys[i])
            torch.cuda.synchronize()
            assert torch.equal(X.cpu(), got[i]), i


def test_rank_one_tucker(L, orc):
    """The smallest Tucker model, multilinear rank (1, 1, 1), and ranks equal
    to the size in one mode only."""
    from oracle import tucker as tk
    shape, iters = (20, 24, 8), 6
    _, Y = _low_rank(shape, 3, 50)
    for ranks in ((1, 1, 1), (20, 2, 1)):
        X, S = _run(L, shape, ranks, iters, Y)
        ref = tk.TuckerState(orc, Y, orc.Params(n1=20, n2=24), ranks)
        ref.iterate(iters)
        assert maxabs(X, ref.X) <= 1e-4, ranks
        assert maxabs(S, ref.st.get("S")) <= 1e-4, ranks
