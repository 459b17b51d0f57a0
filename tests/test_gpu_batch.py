"""Batched uneven cubes (lrstv_batch_*): every cube of a batch follows
Algorithm 1 exactly as a single plan does, so its outputs must equal a
standalone plan's run on the same input bit for bit (the plan made with
LRSTV_FLAG_JACOBI_PER_SLICE, the Jacobi order a batch runs); one cube is also checked
against the FP64 oracle.  The shapes mix slice heights of the persistent
kernel's variants, a transposed slice (n1 < n2) and a cube taller than the
persistent kernel takes (separate Jacobi launch)."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import dev, f32, host, maxabs

pytestmark = pytest.mark.gpu

SHAPES = [(24, 20, 9), (20, 24, 8), (32, 32, 16), (16, 16, 5), (70, 40, 6), (230, 16, 3), (260, 12, 3)]


@pytest.fixture(scope="module")
def L():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_12879_gb300 import lrstv
    lrstv.load()
    return lrstv


def _cube(shape, seed):
    from synthetic import Recipe, make_cube
    rng = np.random.default_rng(seed)
    sigma = float(rng.uniform(0.05, 0.2))
    clean, noisy = make_cube(Recipe(*shape, 3, 6, (sigma, sigma), float(rng.uniform(0.0, 0.3))), seed)
    return f32(noisy)


def _params(L, shape, i, iters, flags=0):
    # per-cube regularisation weights differ; the penalty schedule is shared
    return L.Params.make(shape[0], shape[1], tau=0.001 * (1 + i % 3), alpha=0.1 + 0.05 * i,
                         max_iter=iters, flags=flags)


@pytest.mark.parametrize("warm", [False, True])
def test_batch_equals_single_plans(L, warm):
    import torch
    iters = 6
    flags = L.FLAG_WARM_START if warm else 0
    Ys = [dev(_cube(sh, 100 + i)) for i, sh in enumerate(SHAPES)]
    params = [_params(L, sh, i, iters, flags) for i, sh in enumerate(SHAPES)]
    with L.Batch(SHAPES, params) as b:
        Xs, Ss = b.run(Ys)
        torch.cuda.synchronize()
        for i, sh in enumerate(SHAPES):
            st = b.plan(i).stats()
            assert st.iters == iters and st.jacobi_unconverged == 0
    for i, sh in enumerate(SHAPES):
        # a batch runs each slice's Jacobi sweeps in one CTA: the plan's same order
        with L.Plan(*sh, _params(L, sh, i, iters, flags | L.FLAG_JACOBI_PER_SLICE)) as pl:
            X, S = pl.run(Ys[i])
            torch.cuda.synchronize()
        assert torch.equal(X, Xs[i]), sh
        assert torch.equal(S, Ss[i]), sh


# repeated shapes with equal parameters share a group (packed state, one launch
# per kernel for the group): three and two cubes of float4-stencil shapes, two
# of a scalar-stencil shape (n1 % 4 != 0), two taller than the persistent
# Jacobi takes, two of 145 rows (its 160-row variant); an equal shape with
# another alpha forms a group of its own
GROUPED = [(24, 20, 9), (24, 20, 9), (70, 42, 6), (24, 20, 9), (70, 42, 6), (260, 12, 3),
           (32, 32, 16), (260, 12, 3), (145, 20, 4), (145, 20, 4), (24, 20, 9)]
GROUP_OF = [0, 0, 1, 0, 1, 2, 3, 2, 4, 4, 5]


def _grouped_params(L, iters, flags):
    out = []
    for i, sh in enumerate(GROUPED):
        alpha = 0.15 if i == len(GROUPED) - 1 else 0.1
        out.append(L.Params.make(sh[0], sh[1], tau=0.002, alpha=alpha, max_iter=iters, flags=flags))
    return out


@pytest.mark.parametrize("warm", [False, True])
def test_batch_groups_equal_single_plans(L, warm):
    import torch
    iters = 6
    flags = L.FLAG_WARM_START if warm else 0
    Ys = [dev(_cube(sh, 400 + i)) for i, sh in enumerate(GROUPED)]
    params = _grouped_params(L, iters, flags)
    with L.Batch(GROUPED, params) as b:
        ng, gof = b.groups()
        assert ng == 6 and gof == GROUP_OF
        Xs, Ss = b.run(Ys)
        torch.cuda.synchronize()
        for i in range(len(GROUPED)):
            st = b.plan(i).stats()
            assert st.iters == iters and st.jacobi_unconverged == 0
            assert st.res_inf[0] >= 0.0 and st.res_inf[1] >= 0.0
        # every cube's own residuals, stats and state, not its group's
        single = _grouped_params(L, iters, flags | L.FLAG_JACOBI_PER_SLICE)
        for i, sh in enumerate(GROUPED):
            with L.Plan(*sh, single[i]) as pl:
                X, S = pl.run(Ys[i])
                torch.cuda.synchronize()
                st1, stb = pl.stats(), b.plan(i).stats()
                assert torch.equal(pl.get("E"), b.plan(i).get("E")), sh
            assert torch.equal(X, Xs[i]), (i, sh)
            assert torch.equal(S, Ss[i]), (i, sh)
            assert list(st1.res_inf) == list(stb.res_inf), (i, sh)
            assert st1.jacobi_max_sweeps == stb.jacobi_max_sweeps, (i, sh)


def _spans_per_iteration(L, shapes, iters):
    import torch
    Ys = [dev(_cube(sh, 500 + i)) for i, sh in enumerate(shapes)]
    params = [L.Params.make(sh[0], sh[1], max_iter=iters, flags=L.FLAG_WARM_START)
              for sh in shapes]
    with L.Batch(shapes, params) as b:
        b.init(Ys)
        b.iterate(2)  # past the first E-step, which starts cold
        plans = [b.plan(i) for i in range(len(shapes))]
        for p in plans:
            p.profile_enable(True)
        b.iterate(iters)
        torch.cuda.synchronize()
        total = sum(sum(p.profile_read().launches) for p in plans)
        for p in plans:
            p.profile_enable(False)
    return total / iters


def test_batch_launches_independent_of_cube_count(L):
    # the profiled kernel launches of a batched step depend on the groups
    # (distinct shapes), not on how many cubes each group holds
    two = _spans_per_iteration(L, [(24, 20, 9), (32, 32, 16)], 3)
    many = _spans_per_iteration(L, [(24, 20, 9)] * 5 + [(32, 32, 16)] * 4, 3)
    assert two == many and two > 0


def test_batch_graph_replay(L):
    import torch
    iters = 4
    shapes = SHAPES[:4]
    Ys = [dev(_cube(sh, 200 + i)) for i, sh in enumerate(shapes)]
    eager = L.Batch(shapes, [_params(L, sh, i, iters) for i, sh in enumerate(shapes)])
    graph = L.Batch(shapes, [_params(L, sh, i, iters, L.FLAG_GRAPH) for i, sh in enumerate(shapes)])
    with eager, graph:
        Xe, Se = eager.run(Ys)
        Xg, Sg = graph.run(Ys)
        Xg2, Sg2 = graph.run(Ys, Xg, Sg)  # cached graph replay
        torch.cuda.synchronize()
        for a, b, c in zip(Xe, Xg, Xg2):
            assert torch.equal(a, b) and torch.equal(a, c)


def test_batch_cube_matches_oracle(L, orc):
    iters = 8
    shapes = [(32, 32, 16), (24, 20, 9)]
    Ys = [_cube(sh, 300 + i) for i, sh in enumerate(shapes)]
    with L.Batch(shapes, [L.Params.make(sh[0], sh[1], max_iter=iters) for sh in shapes]) as b:
        Xs, _ = b.run([dev(y) for y in Ys])
        for sh, y, X in zip(shapes, Ys, Xs):
            ost = orc.State(y, orc.Params(n1=sh[0], n2=sh[1]))
            ost.iterate(iters)
            assert maxabs(host(X, sh), ost.X) <= 1e-4


def test_batch_argument_checks(L):
    lib = L.load()
    p = [L.Params.make(8, 8), L.Params.make(8, 8, mu0=0.02)]  # schedules disagree
    dims = (ctypes.c_int * 6)(8, 8, 4, 8, 8, 4)
    h = ctypes.c_void_p()
    assert lib.lrstv_batch_create(2, dims, (L.Params * 2)(*p), ctypes.byref(h)) == 1
    assert lib.lrstv_batch_create(0, dims, (L.Params * 2)(*p), ctypes.byref(h)) == 1
    assert lib.lrstv_batch_destroy(None) == 1
