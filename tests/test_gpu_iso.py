"""GPU parity of the isotropic LRSTV variant (LRSTV_FLAG_ISO_TV, eq. CRSSTV_iso):
the F-update's group threshold of each voxel's three gradient entries, in the
vectorised and the ragged (scalar) F/S/dual kernels, and whole runs against
the FP64 oracle (ORC_FLAG_ISO_TV) at the plain path's bound: 1e-4 max-abs and
0.01 dB MPSNR."""
import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, host3, load_oracle_state, maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def _noisy(shape, seed):
    from synthetic import Recipe, make_cube
    clean, noisy = make_cube(Recipe(*shape, 4, 12, (0.1, 0.1), 0.1), seed)
    return clean, f32(noisy)


@pytest.mark.parametrize("shape", [(32, 32, 16), (37, 29, 11)])
@pytest.mark.parametrize("exact", [False, True])
def test_step_fs_dual_iso(L, orc, shape, exact):
    """One F/S/dual step from an oracle state after 4 isotropic iterations
    (n1 = 32 takes the float4 kernel, n1 = 37 the scalar one)."""
    _, Y = _noisy(shape, 11)
    n1, n2, _ = shape
    oflags = orc.FLAG_ISO_TV | (orc.FLAG_F_THRESH_EXACT if exact else 0)
    lflags = L.FLAG_ISO_TV | (L.FLAG_F_THRESH_EXACT if exact else 0)
    st = orc.State(Y, orc.Params(n1=n1, n2=n2, tau=0.005), flags=oflags)
    st.iterate(4)
    with L.Plan(*shape, L.Params.make(n1, n2, tau=0.005, flags=lflags)) as pl:
        s = load_oracle_state(pl, st)
        s.flags = oflags
        pl.step_fs_dual()
        s.step_f()
        s.step_s()
        s.step_dual()
        F = host3(pl.get("F"), shape)
        G3 = host3(pl.get("G3"), shape)
        for n in range(3):
            assert maxabs(F[n], s.get("F", n)) <= 1e-6
            assert maxabs(G3[n], s.get("G3", n)) <= 2e-6 * s.mu
        assert maxabs(host(pl.get("S"), shape), s.get("S")) <= 1e-6
    # the threshold zeroes whole voxels, and some but not all of them
    Fo = np.stack([s.get("F", n) for n in range(3)])
    zero = np.all(Fo == 0.0, axis=0)
    assert zero.any() and not zero.all()


@pytest.mark.parametrize("shape,iters,flags", [((32, 32, 16), 20, 0), ((37, 29, 11), 15, 0),
                                                ((24, 20, 9), 12, 1), ((64, 64, 31), 30, 32)])
def test_iso_run_matches_oracle(L, orc, shape, iters, flags):
    """Whole isotropic runs; flags adds F_THRESH_EXACT (1) or WARM_START (32)."""
    from synthetic import mpsnr
    clean, Y = _noisy(shape, 3)
    n1, n2, _ = shape
    p = L.Params.make(n1, n2, max_iter=iters, flags=L.FLAG_ISO_TV | flags)
    with L.Plan(*shape, p) as pl:
        X, S, stats = pl.run(dev(Y), stats=True)
        X, S = host(X, shape), host(S, shape)
    ost = orc.State(Y, orc.Params(n1=n1, n2=n2), flags=orc.FLAG_ISO_TV | (flags & 1))
    ost.iterate(iters)
    print(shape, iters, flags, "max-abs", maxabs(X, ost.X), "dMPSNR",
          mpsnr(X, clean) - mpsnr(ost.X, clean))
    assert stats.iters == iters and stats.jacobi_unconverged == 0
    assert maxabs(X, ost.X) <= 1e-4
    assert maxabs(S, ost.get("S")) <= 1e-4
    assert abs(mpsnr(X, clean) - mpsnr(ost.X, clean)) <= 0.01


def test_iso_differs_from_anisotropic(L):
    """The flag reaches the kernel: the same input gives a different F."""
    import torch
    shape = (32, 32, 16)
    _, Y = _noisy(shape, 4)
    outs = []
    for flags in (0, L.FLAG_ISO_TV):
        with L.Plan(*shape, L.Params.make(32, 32, max_iter=3, flags=flags)) as pl:
            pl.run(dev(Y))
            torch.cuda.synchronize()
            outs.append(host3(pl.get("F"), shape))
    assert np.max(np.abs(outs[0] - outs[1])) > 1e-4


@pytest.mark.parametrize("bf16", [False, True])
def test_all_extensions_together(L, orc, bf16):
    """The isotropic F-update, the Tucker L-update and the warm start in one
    plan, with 3xTF32 or 3xBF16 tensor-core GEMMs, against the FP64 reference
    with the isotropic flag, to the 1e-4 bound of whole runs.  For 3xBF16:
    each product term errs by at most 3 * 2^-18 relative (the dropped lo*lo
    term and the halves' rounding), so one Z-solve or t-SVT step errs by about
    1e-5 of its data (measured 4.7e-6 and 1.3e-6); the steps of an ADMM
    iteration are proximal maps and averages (non-expansive), so eight
    iterations add at most 8e-5."""
    from oracle import tucker as tk
    from tests.test_gpu_tucker import _low_rank
    shape, ranks, iters = (24, 20, 9), (3, 3, 3), 8
    _, Y = _low_rank(shape, 3, 61)
    flags = L.FLAG_ISO_TV | L.FLAG_WARM_START | (L.FLAG_BF16X3 if bf16 else 0)
    with L.Plan(*shape, L.Params.make(24, 20, max_iter=iters, flags=flags)) as pl:
        pl.set_tucker(ranks)
        X, S, st = pl.run(dev(Y), stats=True)
        X = host(X, shape)
    assert st.jacobi_unconverged == 0 and st.gemm_errors == 0
    ref = tk.TuckerState(orc, Y, orc.Params(n1=24, n2=20), ranks, flags=orc.FLAG_ISO_TV)
    ref.iterate(iters)
    print("all extensions (bf16x3=%s): max-abs" % bf16, maxabs(X, ref.X))
    assert maxabs(X, ref.X) <= 1e-4


def test_iso_batch_equals_plans(L):
    """A batch of isotropic cubes gives each plan's bits."""
    import torch
    shapes = [(32, 32, 16), (20, 28, 9)]
    Ys = [dev(_noisy(s, 70 + i)[1]) for i, s in enumerate(shapes)]
    p = L.Params.make(32, 32, max_iter=6, flags=L.FLAG_ISO_TV | L.FLAG_WARM_START)
    with L.Batch(shapes, p) as b:
        Xs, _ = b.run(Ys)
        torch.cuda.synchronize()
        got = [x.cpu() for x in Xs]
    p1 = L.Params.make(32, 32, max_iter=6,
                       flags=L.FLAG_ISO_TV | L.FLAG_WARM_START | L.FLAG_JACOBI_PER_SLICE)
    for i, sh in enumerate(shapes):
        with L.Plan(*sh, p1) as pl:
            X, _ = pl.run(Ys[i])
            torch.cuda.synchronize()
            assert torch.equal(X.cpu(), got[i]), i
