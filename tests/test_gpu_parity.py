"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs.

Tolerances: single operators are compared relative to the data's scale at
FP32 rounding level (1e-5 of the largest magnitude for the DFT-based
operators, whose sums run over up to a few hundred terms); whole iterations
use the 1e-4 max-abs / 0.01 dB MPSNR bound on [0, 1]-scaled cubes.
"""
import numpy as np
import pytest

from tests.gpu_util import dev, dev3, f32, host, host3, load_oracle_state, maxabs

pytestmark = pytest.mark.gpu

SHAPES = [(32, 32, 16), (37, 29, 11), (29, 37, 10), (8, 8, 4), (1, 7, 5), (6, 1, 1), (3, 5, 1),
          (70, 65, 9)]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def rnd(shape, seed, scale=1.0):
    return f32(np.random.default_rng(seed).standard_normal(shape) * scale)


# ------------------------------------------------------------ operators ---
@pytest.mark.parametrize("shape", SHAPES)
def test_diff_and_adjoint(L, orc, shape):
    x = rnd(shape, 1)
    g = rnd((3,) + shape, 2)
    w = (0.7, 1.3, 0.4)
    out = host3(L.lrstv_diff(dev(x), shape, w), shape)
    assert maxabs(out, orc.diff(x, w)) <= 2e-6 * max(1.0, np.abs(x).max())
    adj = host(L.lrstv_diff_adjoint(dev3(g), shape, w), shape)
    assert maxabs(adj, orc.diff_adjoint(g, w)) <= 4e-6 * max(1.0, np.abs(g).max())


def test_soft_threshold(L, orc):
    x = rnd((1000,), 3)
    x[:5] = [0.1, -0.1, 0.0, 0.1000001, -0.0999999]
    y = L.lrstv_soft_threshold(dev(x), 0.1).cpu().numpy()
    ref = orc.soft(x, float(np.float32(0.1)))
    assert maxabs(y, ref) <= 1e-7
    assert np.all(y[np.abs(x) <= np.float32(0.1)] == 0)
    assert L.lrstv_soft_threshold(dev(np.zeros(0)), 0.1).numel() == 0


@pytest.mark.parametrize("shape", SHAPES)
def test_zsolve(L, orc, shape):
    T = rnd(shape, 4)
    w = (1.0, 0.6, 1.4)
    for mu in (0.01, 3.7, 1e6):
        Z = host(L.lrstv_zsolve(dev(T), shape, mu, w), shape)
        ref = orc.zsolve(T, mu, w)
        assert maxabs(Z, ref) <= 1e-5 * np.abs(ref).max(), mu


@pytest.mark.parametrize("shape", SHAPES)
def test_tsvt(L, orc, shape):
    A = rnd(shape, 5)
    from tests.test_oracle_pins import bcirc
    sig = np.linalg.svd(bcirc(A), compute_uv=False) if A.size <= 40000 else None
    ts = [0.0, 1.0, 5.0] if sig is None else [0.0, float(np.percentile(sig, 30)),
                                               float(np.percentile(sig, 90)), float(sig.max() * 1.01)]
    for t in ts:
        out, sw = L.lrstv_tsvt(dev(A), shape, t, sweeps=True)
        ref, _ = orc.tsvt(A, t)
        assert sw >= 0, "Jacobi hit its sweep cap"
        assert maxabs(host(out, shape), ref) <= 2e-5 * np.abs(A).max(), t


def test_tsvt_low_rank_and_large(L, orc):
    """A gradient-like cube whose Fourier slices are rank deficient, and a
    slice height above 256 (the widest Jacobi register tile)."""
    rng = np.random.default_rng(6)
    U = rng.standard_normal((40, 3, 6))
    V = rng.standard_normal((3, 24, 6))
    A = f32(np.einsum("irk,rjk->ijk", U, V))
    out = host(L.lrstv_tsvt(dev(A), A.shape, 0.5), A.shape)
    ref, _ = orc.tsvt(A, 0.5)
    assert maxabs(out, ref) <= 2e-5 * np.abs(A).max()
    # slice heights on each side of the kernels' register tiles (208, 256)
    for shape in ((300, 20, 3), (230, 40, 4), (208, 70, 3), (40, 209, 3)):
        B = rnd(shape, 7)
        out = host(L.lrstv_tsvt(dev(B), B.shape, 2.0), B.shape)
        ref, _ = orc.tsvt(B, 2.0)
        assert maxabs(out, ref) <= 2e-5 * np.abs(B).max(), shape


def test_tsvt_and_run_at_the_maximum_slice_height(L, orc):
    """Slice heights of 512, the largest the Jacobi kernels take (either side
    of the slice), for the standalone t-SVT and for whole iterations."""
    assert L.load().lrstv_max_spatial() == 512
    for shape in ((512, 12, 3), (12, 512, 2)):
        B = rnd(shape, 8)
        out = host(L.lrstv_tsvt(dev(B), B.shape, 2.0), B.shape)
        ref, _ = orc.tsvt(B, 2.0)
        assert maxabs(out, ref) <= 2e-5 * np.abs(B).max(), shape
    shape = (512, 16, 4)
    _, Y = _noisy(shape, 9)
    with L.Plan(*shape, L.Params.make(512, 16, max_iter=6)) as pl:
        X, S = pl.run(dev(Y))
        X = host(X, shape)
    ost = orc.State(Y, orc.Params(n1=512, n2=16))
    ost.iterate(6)
    assert maxabs(X, ost.X) <= 1e-4


# Long spectra: the mode-3 DFT kernels stage twiddles in chunks of 64 bands
# (or frequencies), give each thread 48 frequencies (or bands) and each block
# 128 pixels; these shapes cross every one of those boundaries with ragged
# tails (h = 66, 96, 129, 2049; P = 300 and 180 span several pixel tiles), in
# both slice orientations (n1 < n2 transposes the slices), up to the largest
# n3 a plan takes.
LONG_SPECTRA = [(20, 15, 191), (9, 20, 130), (4, 3, 257), (2, 3, 4096)]


def _slice_sigma_percentiles(A, qs):
    """Percentiles of the Fourier-slice singular values (picks thresholds
    that cut some but not all of them; no expected value comes from here)."""
    Ah = np.fft.fft(A.astype(np.float64), axis=2)
    sig = np.concatenate([np.linalg.svd(Ah[:, :, k], compute_uv=False)
                          for k in range(A.shape[2] // 2 + 1)])
    return [float(np.percentile(sig, q)) for q in qs]


@pytest.mark.parametrize("shape", LONG_SPECTRA)
def test_zsolve_long_spectra(L, orc, shape):
    T = rnd(shape, 14)
    w = (1.0, 0.6, 1.4)
    for mu in (0.01, 3.7):
        Z = host(L.lrstv_zsolve(dev(T), shape, mu, w), shape)
        ref = orc.zsolve(T, mu, w)
        err = maxabs(Z, ref)
        print(shape, mu, "zsolve max-abs / max|ref|", err / np.abs(ref).max())
        assert err <= 1e-5 * np.abs(ref).max(), mu


@pytest.mark.parametrize("shape", LONG_SPECTRA)
def test_tsvt_long_spectra(L, orc, shape):
    A = rnd(shape, 15)
    for t in [0.0] + _slice_sigma_percentiles(A, (30, 90)):
        out, sw = L.lrstv_tsvt(dev(A), shape, t, sweeps=True)
        ref, _ = orc.tsvt(A, t)
        err = maxabs(host(out, shape), ref)
        print(shape, t, "tsvt max-abs / max|A|", err / np.abs(A).max())
        assert sw >= 0, "Jacobi hit its sweep cap"
        assert err <= 2e-5 * np.abs(A).max(), t


def test_run_long_spectrum_and_band_limit(L, orc):
    """Whole iterations on a 12x10x191 cube (two frequency groups, two
    frequency chunks, four band groups), against the oracle at the run
    bound; one band more than the largest n3 is a shape error."""
    shape = (12, 10, 191)
    clean, Y = _noisy(shape, 16)
    with L.Plan(*shape, L.Params.make(12, 10, max_iter=5)) as pl:
        X, S = pl.run(dev(Y))
        X, S = host(X, shape), host(S, shape)
    ost = orc.State(Y, orc.Params(n1=12, n2=10))
    ost.iterate(5)
    print("12x10x191 run max-abs", maxabs(X, ost.X), "S", maxabs(S, ost.get("S")))
    assert maxabs(X, ost.X) <= 1e-4
    assert maxabs(S, ost.get("S")) <= 1e-4
    with pytest.raises(L.LrstvError, match="status 2"):
        L.Plan(2, 2, 4097, L.Params.make(2, 2))


# ------------------------------------------------------------ ADMM steps ---
def _noisy(shape, seed):
    from synthetic import Recipe, make_cube
    n1, n2, n3 = shape
    clean, noisy = make_cube(Recipe(n1, n2, n3, 4, 12, (0.1, 0.1), 0.1), seed)
    return clean, f32(noisy)


@pytest.fixture(scope="module")
def mid_state(orc):
    """An oracle state after 4 iterations on a 32x32x16 cube (rounded to f32)."""
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 11)
    st = orc.State(Y, orc.Params(n1=32, n2=32))
    st.iterate(4)
    return shape, st


def _plan(L, shape, **kw):
    n1, n2, n3 = shape
    return L.Plan(n1, n2, n3, L.Params.make(n1, n2, **kw))


def test_step_l_tz(L, orc, mid_state):
    shape, st = mid_state
    with _plan(L, shape) as pl:
        s = load_oracle_state(pl, st)
        pl.step_l_tz()
        s.step_l()
        assert maxabs(host(pl.get("L"), shape), s.get("L")) <= 1e-6
        # T_z of the oracle, written out from its definition (eq. Z_solution)
        w = tuple(s.p[3:6])
        F = np.stack([s.get("F", n) for n in range(3)])
        G3 = np.stack([s.get("G3", n) for n in range(3)])
        T = s.mu * s.get("L") + s.mu * orc.diff_adjoint(F, w) + s.get("G2") - orc.diff_adjoint(G3, w)
        assert maxabs(host(pl.get("TZ"), shape), T) <= 2e-6 * max(1.0, np.abs(T).max())


def test_step_z(L, orc, mid_state):
    shape, st = mid_state
    with _plan(L, shape) as pl:
        s = load_oracle_state(pl, st)
        pl.step_l_tz()
        pl.step_z()
        s.step_l()
        s.step_z()
        assert maxabs(host(pl.get("Z"), shape), s.get("Z")) <= 2e-5


def test_step_fs_dual(L, orc, mid_state):
    shape, st = mid_state
    with _plan(L, shape) as pl:
        s = load_oracle_state(pl, st)
        pl.step_fs_dual()
        s.step_f()
        s.step_s()
        s.step_dual()
        # the multipliers carry a factor mu; compare them relative to mu
        for name, tol in (("S", 1e-6), ("G1", 2e-6 * s.mu), ("G2", 2e-6 * s.mu)):
            assert maxabs(host(pl.get(name), shape), s.get(name)) <= tol, name
        for name, tol in (("F", 1e-6), ("G3", 2e-6 * s.mu)):
            got = host3(pl.get(name), shape)
            for n in range(3):
                assert maxabs(got[n], s.get(name, n)) <= tol, name


def test_step_e(L, orc, mid_state):
    shape, st = mid_state
    with _plan(L, shape) as pl:
        s = load_oracle_state(pl, st)
        pl.step_e()
        s.step_e()
        # the oracle's Gamma4 update belongs to its dual step
        G4 = [s.get("G4", n) + s.mu * (s.get("E", n) - s.get("F", n)) for n in range(3)]
        E = host3(pl.get("E"), shape)
        G = host3(pl.get("G4"), shape)
        for n in range(3):
            assert maxabs(E[n], s.get("E", n)) <= 1e-5
            assert maxabs(G[n], G4[n]) <= 1e-5 * s.mu
        st_ = pl.stats()
        assert st_.jacobi_unconverged == 0 and st_.jacobi_max_sweeps > 0


def test_step_mu(L):
    with _plan(L, (8, 8, 4), mu0=0.5, rho=3.0, mu_max=4.0) as pl:
        pl.init(dev(np.zeros((8, 8, 4))))
        assert pl.mu == (0.5, 0)
        pl.step_mu()
        assert pl.mu == (1.5, 1)
        pl.step_mu()
        assert pl.mu == (4.0, 2)


# ------------------------------------------------------- whole iterations ---
def _run_both(L, orc, shape, iters, seed, flags=0, **kw):
    clean, Y = _noisy(shape, seed)
    n1, n2, n3 = shape
    P = L.Params.make(n1, n2, max_iter=iters, flags=flags, **kw)
    with L.Plan(n1, n2, n3, P) as pl:
        X, S, stats = pl.run(dev(Y), stats=True)
        X, S = host(X, shape), host(S, shape)
    op = orc.Params(n1=n1, n2=n2, **{k: v for k, v in kw.items() if k in ("tau", "alpha", "lam")})
    ost = orc.State(Y, op, flags=flags & 3)
    ost.iterate(iters)
    return clean, X, S, stats, ost


def test_end_to_end_config1(L, orc):
    """32x32x16 synthetic cube, 20 iterations: 1e-4 max-abs, 0.01 dB MPSNR."""
    from synthetic import mpsnr
    clean, X, S, stats, ost = _run_both(L, orc, (32, 32, 16), 20, 1)
    assert maxabs(X, ost.X) <= 1e-4
    assert maxabs(S, ost.get("S")) <= 1e-4
    assert abs(mpsnr(X, clean) - mpsnr(ost.X, clean)) <= 0.01
    assert mpsnr(X, clean) > 25.0
    assert stats.iters == 20 and stats.jacobi_unconverged == 0
    assert abs(stats.mu - ost.mu) <= 1e-6 * ost.mu


@pytest.mark.parametrize("flags", [1, 2])
def test_end_to_end_reading_flags(L, orc, flags):
    clean, X, S, stats, ost = _run_both(L, orc, (24, 20, 9), 12, 5, flags=flags)
    assert maxabs(X, ost.X) <= 1e-4


@pytest.mark.parametrize("shape", [(1, 7, 5), (6, 1, 3), (5, 4, 1), (2, 2, 2), (9, 3, 2)])
def test_end_to_end_degenerate_shapes(L, orc, shape):
    """Whole runs on a single row or column, a single band (one Fourier
    slice, no mode-3 differences to speak of) and the smallest cubes."""
    rng = np.random.default_rng(sum(shape))
    Y = f32(rng.uniform(0.0, 1.0, shape))
    n1, n2, n3 = shape
    with L.Plan(n1, n2, n3, L.Params.make(n1, n2, max_iter=8)) as pl:
        X, S = pl.run(dev(Y))
        X, S = host(X, shape), host(S, shape)
    ost = orc.State(Y, orc.Params(n1=n1, n2=n2))
    ost.iterate(8)
    assert maxabs(X, ost.X) <= 1e-4, shape
    assert maxabs(S, ost.get("S")) <= 1e-4, shape


def test_end_to_end_ragged(L, orc):
    clean, X, S, stats, ost = _run_both(L, orc, (37, 29, 11), 15, 3)
    assert maxabs(X, ost.X) <= 1e-4


def test_graph_replay_matches_eager(L):
    import torch
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 2)
    outs = []
    for flags in (0, L.FLAG_GRAPH):
        with _plan(L, shape, max_iter=6, flags=flags) as pl:
            X, S = pl.run(dev(Y))
            X2, S2 = pl.run(dev(Y))  # graph replay (cached) or a second eager run
            torch.cuda.synchronize()
            assert torch.equal(X, X2) and torch.equal(S, S2)
            outs.append(X.cpu())
    assert torch.equal(outs[0], outs[1])


def test_run_host_matches_device(L):
    import torch
    shape = (20, 24, 7)
    _, Y = _noisy(shape, 4)
    y = np.ascontiguousarray(Y.reshape(-1, order="F").astype(np.float32))
    with _plan(L, shape, max_iter=5) as pl:
        X, S = pl.run(dev(Y))
        Xh = np.empty_like(y)
        Sh = np.empty_like(y)
        st = pl.run_host(y, Xh, Sh, stats=True)
        assert st.iters == 5
        assert np.array_equal(X.cpu().numpy(), Xh) and np.array_equal(S.cpu().numpy(), Sh)
        # pinned host tensors take the same path
        yp = torch.from_numpy(y).pin_memory()
        xp = torch.empty_like(yp).pin_memory()
        sp = torch.empty_like(yp).pin_memory()
        pl.run_host(yp, xp, sp)
        assert np.array_equal(xp.numpy(), Xh)


def test_checkpoint_resume(L):
    """Exporting the state and mu after k iterations and importing it into a
    fresh plan continues the run exactly."""
    import torch
    shape = (16, 12, 6)
    _, Y = _noisy(shape, 8)
    with _plan(L, shape) as a, _plan(L, shape) as b:
        a.init(dev(Y))
        a.iterate(3)
        saved = {n: a.get(n) for n in ("Y", "L", "Z", "S", "G1", "G2", "F", "E", "G3", "G4")}
        mu, it = a.mu
        a.iterate(2)
        for n, v in saved.items():
            b.set(n, v)
        b.set_mu(mu, it)
        b.iterate(2)
        torch.cuda.synchronize()
        assert torch.equal(a.get("L"), b.get("L"))
        assert a.mu == b.mu


def test_constant_cube_is_fixed_point(L):
    shape = (10, 9, 5)
    Y = np.full(shape, 0.37)
    with _plan(L, shape, max_iter=5) as pl:
        X, S = pl.run(dev(Y))
        assert maxabs(host(X, shape), Y) <= 1e-6
        assert float(S.abs().max()) == 0.0


def test_nonfinite_input_is_reported(L):
    shape = (8, 8, 4)
    Y = np.zeros(shape)
    Y[1, 2, 3] = np.nan
    with _plan(L, shape, max_iter=2, flags=L.FLAG_STRICT) as pl:
        with pytest.raises(L.LrstvError) as e:
            pl.run(dev(Y), stats=True)
        assert e.value.code == 6


def test_denoise_one_shot(L, orc):
    shape = (16, 16, 8)
    _, Y = _noisy(shape, 9)
    X, S, st = L.lrstv_denoise(dev(Y), shape, L.Params.make(16, 16, max_iter=4))
    ost = orc.State(Y, orc.Params(n1=16, n2=16))
    ost.iterate(4)
    assert maxabs(host(X, shape), ost.X) <= 1e-4
    assert st.iters == 4


def test_tensor_core_gemm_matches_simt(L, orc, mid_state):
    """The spatial DFT and SVT-reconstruction GEMMs on the tensor cores
    (tcgen05, 3xTF32) against the FP32 SIMT kernel, on the same state."""
    shape, st = mid_state
    outs = {}
    for flags in (0, L.FLAG_SIMT_GEMM):
        with _plan(L, shape, flags=flags) as pl:
            load_oracle_state(pl, st)
            pl.step_l_tz()
            pl.step_z()
            pl.step_fs_dual()
            pl.step_e()
            s = pl.stats()
            assert s.gemm_errors == 0
            outs[flags] = (host(pl.get("Z"), shape), host3(pl.get("E"), shape))
    z_tc, e_tc = outs[0]
    z_si, e_si = outs[L.FLAG_SIMT_GEMM]
    # 3xTF32 carries ~2^-21 per product; FP32 sums on both sides
    assert maxabs(z_tc, z_si) <= 2e-6 * max(1.0, np.abs(z_si).max())
    assert maxabs(e_tc, e_si) <= 2e-6 * max(1.0, np.abs(e_si).max())


@pytest.mark.parametrize("shape", [(200, 200, 4), (130, 70, 5), (37, 29, 11)])
def test_tensor_core_zsolve_shapes(L, orc, shape):
    """Tile edges of the tensor-core GEMM (128-row and 64-column tiles, ragged
    K) through a plan's Z-step, against the oracle's solve of the same T_z."""
    n1, n2, n3 = shape
    rng = np.random.default_rng(21)
    with _plan(L, shape) as pl:
        pl.init(dev(np.zeros(shape)))
        T = f32(rng.standard_normal(shape))
        pl.set("TZ", dev(T))
        pl.step_z()
        mu, _ = pl.mu
        ref = orc.zsolve(T, mu)
        assert maxabs(host(pl.get("Z"), shape), ref) <= 1e-5 * np.abs(ref).max()
        assert pl.stats().gemm_errors == 0


@pytest.mark.parametrize("shape", LONG_SPECTRA + [(37, 29, 11), (29, 37, 10)])
@pytest.mark.parametrize("bf16", [False, True])
def test_tensor_core_mode3_dfts(L, orc, shape, bf16):
    """The mode-3 (spectral) DFTs on the tensor cores, through a plan's Z-step
    and E-step, against the oracle's Z-solve and t-SVT: long spectra (K and N
    chunks with ragged tails: h = 66, 96, 129, 2049) and both slice
    orientations (n1 < n2 writes and reads the transposed, conjugated
    slices).  Bounds: 3xTF32 as the SIMT kernels' (1e-5 of the Z-solve's
    largest value, 2e-5 of max|F| for the t-SVT); 3xBF16 2e-4, the
    mixed-precision step bound (about 1e-5 relative per product term)."""
    n1, n2, n3 = shape
    rng = np.random.default_rng(31)
    flags = L.FLAG_BF16X3 if bf16 else 0
    tz, te = (2e-4, 2e-4) if bf16 else (1e-5, 2e-5)
    with _plan(L, shape, flags=flags) as pl:
        pl.init(dev(np.zeros(shape)))
        T = f32(rng.standard_normal(shape))
        pl.set("TZ", dev(T))
        pl.step_z()
        mu, _ = pl.mu
        ref = orc.zsolve(T, mu)
        err = maxabs(host(pl.get("Z"), shape), ref)
        print(shape, bf16, "Z-step max-abs / max|ref|", err / np.abs(ref).max())
        assert err <= tz * np.abs(ref).max()
        # E-step with Gamma4 = 0: E_n = t-SVT(F_n, alpha / mu), Gamma4_n = mu (E_n - F_n)
        F = [f32(rng.standard_normal(shape)) for _ in range(3)]
        t = _slice_sigma_percentiles(F[0], (60,))[0]
        mu_e = 0.2 / t  # the plan's alpha is 0.2
        pl.set_mu(mu_e, 5)
        pl.set("F", dev3(F))
        pl.set("G4", dev3([np.zeros(shape)] * 3))
        pl.step_e()
        s = pl.stats()
        assert s.gemm_errors == 0 and s.jacobi_unconverged == 0
        E = host3(pl.get("E"), shape)
        G4 = host3(pl.get("G4"), shape)
        tf = float(np.float32(float(np.float32(0.2)) / mu_e))  # the plan's alpha / mu, rounded
        for n in range(3):
            want, _ = orc.tsvt(F[n], tf)
            err = maxabs(E[n], want)
            print(shape, bf16, n, "E-step max-abs / max|F|", err / np.abs(F[n]).max())
            assert err <= te * np.abs(F[n]).max(), n
            assert maxabs(G4[n], mu_e * (E[n] - F[n])) <= 1e-5 * mu_e * np.abs(F[n]).max(), n


def test_dft_engines_agree(L, orc):
    """A whole run with the mode-3 DFTs on the SIMT kernels (LRSTV_FLAG_SIMT_DFT)
    and one with them on the tensor cores: both within the run bound of the
    oracle, and within 2e-6 of each other (3xTF32 against FP32 direct sums)."""
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 19)
    outs = []
    for flags in (0, L.FLAG_SIMT_DFT):
        with _plan(L, shape, max_iter=12, flags=flags | L.FLAG_WARM_START) as pl:
            X, _ = pl.run(dev(Y))
            outs.append(host(X, shape))
    ost = orc.State(Y, orc.Params(n1=32, n2=32))
    ost.iterate(12)
    for X in outs:
        assert maxabs(X, ost.X) <= 1e-4
    assert maxabs(outs[0], outs[1]) <= 2e-6 * max(1.0, np.abs(outs[1]).max())


@pytest.mark.parametrize("shape", [(32, 32, 16), (70, 65, 9), (29, 37, 10), (200, 64, 4),
                                   (150, 48, 6)])
def test_jacobi_schedules_agree(L, orc, shape):
    """The task-graph Jacobi (the default: every SM takes panel-pair tasks of
    any slice) and one CTA per slice (LRSTV_FLAG_JACOBI_PER_SLICE), each with
    32- and 16-column panels (LRSTV_FLAG_JACOBI_PANEL16), visit every column
    pair once per sweep in different orders: whole warm-started runs of all
    four are within the run bound of the oracle.  Shapes with one, three and
    two column panels (odd and even counts: the tournament's one or two empty
    players), a transposed slice, and slices of 129-160 rows (the 160-row
    variant)."""
    n1, n2, n3 = shape
    _, Y = _noisy(shape, 23)
    iters = 10
    outs = []
    for flags in (L.FLAG_WARM_START, L.FLAG_WARM_START | L.FLAG_JACOBI_PER_SLICE,
                  L.FLAG_WARM_START | L.FLAG_JACOBI_PANEL16,
                  L.FLAG_WARM_START | L.FLAG_JACOBI_PER_SLICE | L.FLAG_JACOBI_PANEL16):
        with _plan(L, shape, max_iter=iters, flags=flags) as pl:
            X, S, st = pl.run(dev(Y), stats=True)
            assert st.jacobi_unconverged == 0
            outs.append(host(X, shape))
    ost = orc.State(Y, orc.Params(n1=n1, n2=n2))
    ost.iterate(iters)
    for X in outs:
        assert maxabs(X, ost.X) <= 1e-4
