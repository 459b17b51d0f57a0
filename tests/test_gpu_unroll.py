"""GPU parity of the unrolled, differentiable iteration (lrstv_unroll_*).

The forward pass with the plain solver's scalars must equal a plan's run bit
for bit (same kernels, same arithmetic).  With free per-iteration scalars the
forward pass is compared with the FP64 reference (oracle/adjoint.py) at the
iteration's 1e-4 max-abs bound, and the backward pass -- fed the same dLoss/dX
as the reference -- is compared gradient by gradient.

Gradient tolerance: every gradient is a sum over the cube of products of
FP32 iterates (relative error ~1e-6 after a few iterations) with adjoint
values, so its error is bounded by ~1e-6 times the sum of the magnitudes of
its terms.  The scalars' gradients are held to 1e-4 of the largest gradient
of the same scalar (measured: at most 7e-6), dY to 1e-5 of its largest entry
on the small cubes (measured: 3e-7); a dropped term, sign or factor changes a
gradient by O(1) of its own size.  At 64x64x31 x 10 iterations some voxels sit
within FP32 rounding of a soft threshold (see _check_dY).
"""
import numpy as np
import pytest

from tests.gpu_util import f32, maxabs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def _cubes(shape, B, seed):
    from synthetic import Recipe, make_cube
    out = []
    for b in range(B):
        clean, noisy = make_cube(Recipe(*shape, 3, 6, (0.1, 0.1), 0.1), seed + b)
        out.append((f32(clean), f32(noisy)))
    return out


def _to_dev(cubes):
    """list of (n1, n2, n3) arrays -> (B, n3, n2, n1) float32 CUDA tensor."""
    import torch
    a = np.stack([np.asarray(c, np.float32).transpose(2, 1, 0) for c in cubes])
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _to_host(t):
    """(B, n3, n2, n1) tensor -> list of float64 (n1, n2, n3) arrays."""
    a = t.detach().cpu().numpy().astype(np.float64)
    return [a[b].transpose(2, 1, 0) for b in range(a.shape[0])]


def _plain_theta(p, K):
    mu, out = float(p.mu0), []
    for _ in range(K):
        out.append([float(p.tau), float(p.alpha), float(p.lam), mu])
        mu = min(float(p.rho) * mu, float(p.mu_max))
    return np.array(out)


def _free_theta(K):
    """Scalars at which every threshold of the iteration cuts part of its
    input: about half the F entries, half the S entries (after the first
    iteration) and 2-25% of the singular values of the Fourier slices are
    kept, so every branch of the adjoint carries weight."""
    return np.array([[0.02 * (1 + 0.3 * k), 0.4 + 0.1 * k, 0.12 * 1.4 ** k, 1.4 ** k]
                     for k in range(K)])


@pytest.mark.parametrize("shape", [(24, 20, 9), (20, 24, 8)])
@pytest.mark.parametrize("warm", [False, True])
def test_forward_equals_plan_bitwise(L, shape, warm):
    import torch
    K, B = 4, 2
    cubes = _cubes(shape, B, 40)
    Y = _to_dev([c[1] for c in cubes])
    flags = L.FLAG_WARM_START if warm else 0
    p = L.Params.make(shape[0], shape[1], max_iter=K, flags=flags)
    with L.Unroll(shape, B, K, flags=flags) as u:
        X = u.forward(Y, _plain_theta(p, K))
        assert u.stats() == (0, 0)
    for b in range(B):
        with L.Plan(*shape, p) as pl:
            Xp, _ = pl.run(Y[b].reshape(-1).contiguous())
            torch.cuda.synchronize()
        assert torch.equal(Xp, X[b].reshape(-1)), b


def _oracle(cube, thetas, dX):
    from oracle import adjoint as adj
    X, tape = adj.unrolled_forward(cube, thetas)
    g_theta, g_Y = adj.unrolled_backward(tape, dX)
    return X, g_theta, g_Y


def _check_theta(g_gpu, g_orc, rtol=1e-4):
    scale = np.max(np.abs(g_orc), axis=0)
    err = np.max(np.abs(g_gpu - g_orc), axis=0)
    print("dtheta error / scale per column:", err / np.where(scale > 0, scale, 1.0))
    assert np.all(scale > 0), "every scalar must carry gradient"
    assert np.all(err <= rtol * scale), (err / scale, g_gpu, g_orc)


def _check_dY(dY_gpu, dY_orc, rtol=2e-3, max_out=None):
    """dY voxel by voxel.  Each side takes the soft-threshold decisions of
    the forward pass in its own precision, so a voxel whose threshold input
    lies within FP32 rounding of the threshold may take the other branch on
    the GPU and move the gradient near it by up to its own size.  The bound:
    the whole field within rtol in the 2-norm, and at most one voxel in a
    thousand outside rtol of the largest entry."""
    d = np.abs(np.asarray(dY_gpu) - np.asarray(dY_orc))
    top = np.max(np.abs(dY_orc))
    l2 = np.linalg.norm(d) / np.linalg.norm(dY_orc)
    out = int(np.sum(d > rtol * top))
    print(f"dY: max error / max {np.max(d) / top:.3e}, 2-norm relative {l2:.3e}, "
          f"{out} of {d.size} voxels outside {rtol} of max")
    assert l2 <= rtol
    assert out <= (d.size // 1000 if max_out is None else max_out)


@pytest.mark.parametrize("shape", [(16, 12, 7), (12, 16, 6)])
def test_unroll_matches_oracle(L, shape):
    # E of iteration k reaches L first in iteration k + 3, so K = 5 lets the
    # t-SVT adjoint of the first two iterations carry gradient
    K, B = 5, 2
    cubes = _cubes(shape, B, 60)
    Y = _to_dev([c[1] for c in cubes])
    theta = _free_theta(K)
    rng = np.random.default_rng(3)
    dXs = [f32(rng.standard_normal(shape) / np.prod(shape)) for _ in range(B)]
    with L.Unroll(shape, B, K) as u:
        X = u.forward(Y, theta)
        assert u.stats() == (0, 0)
        dth, dY = u.backward(_to_dev(dXs))
        dth = dth.cpu().numpy()
        dYh = _to_host(dY)
        Xh = _to_host(X)
    g_tot = np.zeros((K, 4))
    for b in range(B):
        Xo, g_o, dY_o = _oracle(cubes[b][1], theta, dXs[b])
        assert maxabs(Xh[b], Xo) <= 1e-4
        g_tot += g_o
        _check_dY(dYh[b], dY_o, rtol=1e-5, max_out=0)
    _check_theta(dth, g_tot)


def test_unroll_simt_gemm_agrees(L):
    """The tensor-core and SIMT GEMM paths give the same gradients to FP32
    accuracy (the backward's own GEMMs are SIMT in both)."""
    shape, K, B = (16, 16, 8), 3, 2
    cubes = _cubes(shape, B, 70)
    Y = _to_dev([c[1] for c in cubes])
    theta = _free_theta(K)
    dX = _to_dev([f32(np.full(shape, 1.0 / np.prod(shape))) for _ in range(B)])
    out = []
    for flags in (0, L.FLAG_SIMT_GEMM):
        with L.Unroll(shape, B, K, flags=flags) as u:
            X = u.forward(Y, theta)
            dth, dY = u.backward(dX)
            out.append((X.cpu().numpy(), dth.cpu().numpy(), dY.cpu().numpy()))
    (X0, t0, y0), (X1, t1, y1) = out
    assert np.max(np.abs(X0 - X1)) <= 1e-5
    assert np.max(np.abs(t0 - t1)) <= 1e-3 * np.max(np.abs(t1))
    assert np.max(np.abs(y0 - y1)) <= 1e-3 * np.max(np.abs(y1))


@pytest.mark.parametrize("flags", ["cold", "warm", "warm_per_slice"])
def test_unroll_recompute_bitwise(L, flags):
    """LRSTV_FLAG_UNROLL_RECOMPUTE keeps one slot of SVD factors and reruns each
    E-update's SVDs from the checkpointed states in the backward pass: the
    same kernels on the same inputs, so the iterate and dY equal the storing
    handle's bit for bit, twice in a row (a warm start rewrites the kept V
    slots with the same bits), and the scalars' gradients up to the order of
    their FP64 atomic sums, in a smaller arena."""
    import torch
    fl = {"cold": 0, "warm": L.FLAG_WARM_START,
          "warm_per_slice": L.FLAG_WARM_START | L.FLAG_JACOBI_PER_SLICE}[flags]
    shape, K, B = (24, 20, 9), 5, 2
    cubes = _cubes(shape, B, 80)
    Y = _to_dev([c[1] for c in cubes])
    theta = _free_theta(K)
    rng = np.random.default_rng(5)
    dX = _to_dev([f32(rng.standard_normal(shape) / np.prod(shape)) for _ in range(B)])
    res, sizes = [], []
    for extra in (0, L.FLAG_UNROLL_RECOMPUTE):
        with L.Unroll(shape, B, K, flags=fl | extra) as u:
            sizes.append(u.nbytes)
            X = u.forward(Y, theta)
            runs = []
            for _ in range(2):
                dth, dY = u.backward(dX)
                runs.append((dth.cpu().numpy(), dY.cpu().numpy()))
            assert u.stats() == (0, 0)
            res.append((X.cpu().numpy(), runs))
    (X0, r0), (X1, r1) = res
    assert np.array_equal(X0, X1)
    # dY is bitwise; the scalars' gradients are FP64 sums whose block partials
    # arrive by atomics in no fixed order, so two runs of one handle already
    # differ in the last bits: they are held to 1e-12 of each column's largest
    top = np.max(np.abs(r0[0][0]), axis=0) + 1e-300
    for t, y in r0[1:] + r1:
        assert np.array_equal(y, r0[0][1])
        assert np.all(np.abs(t - r0[0][0]) <= 1e-12 * top)
    assert np.count_nonzero(r0[0][0]) >= 8
    # factor slots: W and sigma for K - 1 iterations, V too without a warm start
    n1, n2, n3 = shape
    ns, nc = 3 * B * (n3 // 2 + 1), min(n1, n2)
    saved = (K - 1) * ns * (n1 * n2 * 8 + nc * 8) + (0 if fl else (K - 1) * ns * nc * nc * 8)
    assert sizes[0] - sizes[1] >= saved - 3 * 256  # up to 256 bytes of alignment a field
    torch.cuda.synchronize()


def test_unroll_argument_checks(L):
    import ctypes
    import torch
    lib = L.load()
    h = ctypes.c_void_p()
    w = (ctypes.c_float * 3)(1, 1, 1)
    assert lib.lrstv_unroll_create(8, 8, 4, 0, 2, w, 0, ctypes.byref(h)) == 1
    assert lib.lrstv_unroll_create(8, 8, 4, 1, 0, w, 0, ctypes.byref(h)) == 1
    assert lib.lrstv_unroll_create(8, 8, 4, 1, 2, w, 1, ctypes.byref(h)) == 1  # F_THRESH_EXACT
    assert lib.lrstv_unroll_create(8, 8, 4000, 1, 2, w, 0, ctypes.byref(h)) == 0
    lib.lrstv_unroll_destroy(h)
    assert lib.lrstv_unroll_create(600, 8, 4, 1, 2, w, 0, ctypes.byref(h)) == 2
    with L.Unroll((8, 8, 4), 1, 2) as u:
        Y = torch.rand(1, 4, 8, 8, device="cuda")
        dX = torch.ones_like(Y)
        with pytest.raises(L.LrstvError, match="status 7"):
            u.backward(dX)
        for bad in ([[1e-3, 0.2, 0.1, 0.0]] * 2, [[-1e-3, 0.2, 0.1, 1.0]] * 2,
                    [[np.nan, 0.2, 0.1, 1.0]] * 2):
            with pytest.raises(L.LrstvError, match="status 1"):
                u.forward(Y, bad)
        with pytest.raises(ValueError):
            u.forward(Y, [[1e-3, 0.2, 0.1, 1.0]])


def test_autograd_module_matches_direct_calls(L):
    import torch
    from paper_2204_12879_gb300.unrolled import UnrolledLRSTV
    shape, B, K = (16, 16, 8), 2, 3
    cubes = _cubes(shape, B, 80)
    Y = _to_dev([c[1] for c in cubes]).requires_grad_(True)
    clean = _to_dev([c[0] for c in cubes])
    m = UnrolledLRSTV(*shape, batch=B, iters=K)
    X = m(Y)
    loss = ((X - clean) ** 2).mean()
    loss.backward()
    g_log = m.log_theta.grad.clone()
    # the same through the handle directly
    theta = m.theta().detach()
    dX = (2.0 * (X.detach() - clean) / X.numel()).contiguous()
    X2 = m.handle.forward(Y.detach(), theta.numpy())
    assert torch.equal(X2, X.detach())
    dth, dY = m.handle.backward(dX)
    # torch forms dLoss/dX in its own operation order: equal up to FP32 rounding
    want = dth.cpu() * theta
    assert torch.allclose(g_log, want, rtol=1e-4, atol=1e-6 * float(want.abs().max()))
    assert torch.allclose(Y.grad, dY, rtol=1e-4, atol=1e-6 * float(dY.abs().max()))
    # one optimiser step keeps every scalar positive and changes the loss
    opt = torch.optim.Adam(m.parameters(), lr=0.05)
    opt.step()
    assert torch.all(m.theta() > 0)
    with torch.no_grad():
        loss2 = ((m(Y.detach()) - clean) ** 2).mean()
    assert float(loss2) != float(loss)


@pytest.mark.slow
def test_unroll_training_shape_cube0_matches_oracle(L):
    """The 64x64x31 batch-8, 10-iteration configuration of the unrolled
    solver: forward + backward through the library; the gradient of a loss on
    cube 0 alone is compared with the FP64 reference."""
    import torch
    shape, B, K = (64, 64, 31), 8, 10
    cubes = _cubes(shape, B, 90)
    Y = _to_dev([c[1] for c in cubes])
    from paper_2204_12879_gb300.unrolled import default_theta
    theta = np.array(default_theta(64, 64, K))  # where a training run starts
    dX0 = f32(2.0 * (cubes[0][1] - cubes[0][0]) / np.prod(shape))
    dXs = [dX0] + [np.zeros(shape, np.float32)] * (B - 1)
    with L.Unroll(shape, B, K, flags=L.FLAG_WARM_START) as u:
        X = u.forward(Y, theta)
        assert u.stats() == (0, 0)
        dth, dY = u.backward(_to_dev(dXs))
        torch.cuda.synchronize()
        dth = dth.cpu().numpy()
        dYh = _to_host(dY)
        Xh = _to_host(X)
    assert all(np.all(np.isfinite(x)) for x in Xh)
    Xo, g_o, dY_o = _oracle(cubes[0][1], theta, dX0)
    assert maxabs(Xh[0], Xo) <= 1e-4
    _check_theta(dth, g_o)
    _check_dY(dYh[0], dY_o)
    for b in range(1, B):
        assert np.max(np.abs(dYh[b])) == 0.0
