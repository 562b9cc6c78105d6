"""Many independent problems in one chase_solve_batch call, and warm starts
along a sequence of perturbed matrices (A_{t+1} = A_t + 1e-3 E_t, ||E_t||_2 = 1).

The batch advances all problems through Alg. 2 in lockstep: their
reduced-precision filter phases run as grouped tensor-core launches (one per
degree step for all problems, captured in a CUDA graph), and so do their FP64
filter phases when the FP64 products are the tensor-core ones (per degree step
one grouped digit-slicing launch and one grouped product launch); the other
phases run on each problem's own context and stream from a host thread pool. Every tile of a
grouped launch is computed exactly as in the problem's own launch and every
reduction has a fixed order, so the batched results must equal the
one-at-a-time results bit for bit. The tensor-core filter's raster order is
picked by timing on first use; the order cannot change a result, which the
repeated-filter test checks.
"""
import numpy as np
import pytest

from synth import Problem, complex_normal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x, lib):
    return lib.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def batch_problem(N, seed):
    # nev = ceil(N/20), nex = ceil(N/40), uniform spectrum, 8 reflectors
    return Problem(N=N, nev=-(-N // 20), nex=-(-N // 40), spectrum="uniform", lo=0.0,
                   hi=10.0, reflectors=8, seed=seed)


def unit_hermitian(N, seed):
    Z = complex_normal(seed, 95, N * N).reshape(N, N)
    E = 0.5 * (Z + Z.conj().T)
    return E / np.abs(np.linalg.eigvalsh(E)).max()


@pytest.mark.parametrize("tensor,precision", [(0, 0), (1, 1), (0, 1), (1, 0)])
def test_batch_equals_single_solves(lib, tensor, precision):
    sizes = [256, 700, 384, 1000, 300]
    probs = [batch_problem(N, 40 + k) for k, N in enumerate(sizes)]
    As = [dev(p.matrix(), lib) for p in probs]

    def run(batched):
        ctxs, Vs, rz, rs = [], [], [], []
        streams = [torch.cuda.Stream() for _ in probs]
        for p, s in zip(probs, streams):
            prm = lib.default_params(p.N, p.nev, p.nex, fp64_tensor=tensor, precision=precision)
            ctxs.append(lib.Context(prm, s))
            Vs.append(dev(p.start_block(), lib))
            rz.append(torch.zeros(p.ne, dtype=torch.float64, device="cuda"))
            rs.append(torch.zeros(p.ne, dtype=torch.float64, device="cuda"))
        Q0 = [dev(p.lanczos_start(), lib) for p in probs]
        torch.cuda.synchronize()
        if batched:
            stats, status = lib.solve_batch(ctxs, As, Vs, rz, rs, lanczos_starts=Q0, threads=3)
        else:
            stats = [cx.chase_solve(A, V, r, s, lanczos_start=q)
                     for cx, A, V, r, s, q in zip(ctxs, As, Vs, rz, rs, Q0)]
            status = [st["status"] for st in stats]
        torch.cuda.synchronize()
        for cx in ctxs:
            cx.close()
        return ([v.cpu().numpy() for v in Vs], [r.cpu().numpy() for r in rz],
                [r.cpu().numpy() for r in rs], stats, status)

    Vb, rzb, rsb, stb, sb = run(True)
    Vs, rzs, rss, sts, ss = run(False)
    assert sb == ss == [0] * len(probs)
    for k, p in enumerate(probs):
        assert np.array_equal(rzb[k], rzs[k]), k
        assert np.array_equal(rsb[k], rss[k]), k
        assert np.array_equal(Vb[k], Vs[k]), k
        assert stb[k]["matvecs"] == sts[k]["matvecs"]
        lam = p.eigenvalues()[:p.nev]
        assert np.abs(rzb[k][:p.nev] - lam).max() <= 1e-10 * p.norm2()


def test_warm_start_sequence(lib):
    p = batch_problem(800, 77)
    A0 = p.matrix()
    Ad = dev(A0, lib)
    prm = lib.default_params(p.N, p.nev, p.nex)
    with lib.Context(prm) as cx:
        V = dev(p.start_block(), lib)
        rz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        rs = torch.zeros_like(rz)
        cold0 = cx.chase_solve(Ad, V, rz, rs)
        A = A0
        for t in range(3):
            A = A + 1e-3 * unit_hermitian(p.N, 500 + t)
            Ad = dev(A, lib)
            Vc = dev(p.start_block(), lib)
            cold = cx.chase_solve(Ad, Vc, rz, rs)
            warm = cx.chase_solve(Ad, V, rz, rs)  # V: the previous step's Ritz vectors
            lam = np.linalg.eigvalsh(A)[:p.nev]
            nA = np.abs(np.linalg.eigvalsh(A)).max()
            assert np.abs(rz.cpu().numpy()[:p.nev] - lam).max() <= 1e-10 * nA
            print(f"step {t}: matvecs cold {cold['matvecs']} warm {warm['matvecs']} "
                  f"(first cold solve {cold0['matvecs']})")
            assert warm["matvecs"] < cold["matvecs"]


def test_mixed_filter_independent_of_tuned_raster_order(lib):
    """The first mixed filter call for a shape times the kernel's raster orders
    and keeps the fastest; a second call (cached order) and a fresh context give
    bit-identical results."""
    p = batch_problem(2600, 61)
    A = dev(p.matrix(), lib)
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    c, e, mu1 = (b_sup + lam[p.ne - 1]) / 2, (b_sup - lam[p.ne - 1]) / 2, lam[0]
    degs = np.full(p.ne, 12, dtype=np.int32)
    outs = []
    for _ in range(2):
        with lib.Context(lib.default_params(p.N, p.nev, p.nex,
                                            precision=lib.CHASE_MIXED_BF16X3)) as ctx:
            for _ in range(2):
                V = dev(p.start_block(), lib)
                ctx.chase_filter(A, V, p.ne, degs, c, e, mu1, precision=lib.CHASE_MIXED_BF16X3)
                outs.append(V.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])

