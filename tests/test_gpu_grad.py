"""Gradients through the filter and through the lowest eigenpairs: the CUDA
adjoints (chase_filter_vjp, chase_eig_vjp and the autograd Functions over
them) against the FP64 oracle's gradients and central finite differences.

Tolerances: the filter adjoint is a sequence of FP64 products like the filter
itself, so it matches the oracle to 1e-12 of the largest entry (tensor-core FP64
products: deg * 2^-40). The eigenpair adjoint starts from Ritz pairs converged
to 1e-10 ||A|| and solves the complement part by CG to 1e-10, so it matches the
exact gradient to about (1e-10 ||A|| / gap) relative; the bar is 1e-6 relative
(the gradient tolerance of the differentiation workload); measured values are printed.
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from oracle import grad_oracle as G
from synth import Problem, complex_normal, config_problem, uniform01

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev(x, lib):
    return lib.colmajor(torch.from_numpy(np.asfortranarray(x)).cuda())


def empty_cm(n, m):
    return torch.empty((m, n), dtype=torch.complex128, device="cuda").mT


def rand_herm(n, seed, stream=90):
    Z = complex_normal(seed, stream, n * n).reshape(n, n)
    return 0.5 * (Z + Z.conj().T)


def rand_c(shape, seed, stream=91):
    return complex_normal(seed, stream, int(np.prod(shape))).reshape(shape)


def filter_params(p):
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    return (b_sup + lam[p.ne - 1]) / 2, (b_sup - lam[p.ne - 1]) / 2, lam[0]


# ------------------------------------------------------------- filter VJP
@pytest.mark.parametrize("N,n,deg,ckpt,tensor", [
    (300, 7, 8, 0, 0), (300, 7, 8, 1, 0), (300, 7, 8, 8, 0), (257, 13, 20, 5, 0),
    (129, 1, 3, 2, 0), (400, 33, 20, 5, 1)])
def test_filter_vjp_against_oracle(lib, N, n, deg, ckpt, tensor):
    p = Problem(N=N, nev=n, nex=max(2, n // 3), spectrum="uniform", lo=-1.0, hi=4.0,
                reflectors=5, seed=N + deg)
    A, V = p.matrix(), rand_c((N, n), N)
    Yb = rand_c((N, n), N + 1)
    c, e, mu1 = filter_params(p)
    Ab_o, Vb_o = G.filter_vjp(A, V, deg, c, e, mu1, Yb)
    prm = lib.default_params(N, n, 0, fp64_tensor=tensor)
    with lib.Context(prm) as ctx:
        Ab, Vb = empty_cm(N, N), empty_cm(N, n)
        ctx.chase_filter_vjp(dev(A, lib), dev(V, lib), n, deg, c, e, mu1, dev(Yb, lib), Ab, Vb,
                             checkpoint=ckpt)
        Ab, Vb = Ab.cpu().numpy(), Vb.cpu().numpy()
    ea = np.abs(Ab - Ab_o).max() / np.abs(Ab_o).max()
    ev = np.abs(Vb - Vb_o).max() / np.abs(Vb_o).max()
    print(f"N={N} n={n} deg={deg} ckpt={ckpt} tensor={tensor}: Abar {ea:.2e}, Vbar {ev:.2e}")
    tol = deg * 2.0 ** -40 if tensor else 1e-12
    assert ea <= tol and ev <= tol
    assert np.abs(Ab - Ab.conj().T).max() == 0.0  # exactly Hermitian


def test_filter_autograd_finite_differences(lib):
    from paper_2309_15595_gb300.autograd import chebyshev_filter

    N, n, deg = 200, 5, 10
    p = Problem(N=N, nev=n, nex=3, spectrum="uniform", lo=0.0, hi=3.0, reflectors=4, seed=11)
    A0, V0, W = p.matrix(), rand_c((N, n), 12), rand_c((N, n), 13)
    c, e, mu1 = filter_params(p)
    At = torch.from_numpy(A0).cuda().requires_grad_(True)
    Vt = torch.from_numpy(V0).cuda().requires_grad_(True)
    Wt = torch.from_numpy(W).cuda()
    Y = chebyshev_filter(At, Vt, deg, c, e, mu1, checkpoint=3)
    loss = torch.real(torch.sum(Wt.conj() * Y))
    loss.backward()
    Ag, Vg = At.grad.cpu().numpy(), Vt.grad.cpu().numpy()

    def L(Am, Vm):
        return float(np.real(np.sum(W.conj() * O.chebyshev_filter(Am, Vm, [deg] * n, c, e, mu1))))

    h = 1e-6
    for k in range(6):
        E, dV = rand_herm(N, 500 + k), rand_c((N, n), 600 + k)
        fd = (L(A0 + h * E, V0 + h * dV) - L(A0 - h * E, V0 - h * dV)) / (2 * h)
        an = float(np.real(np.sum(Ag.conj() * E) + np.sum(Vg.conj() * dV)))
        assert abs(fd - an) <= 1e-6 * abs(an), (k, fd, an)


# ----------------------------------------------------------- eigenpair VJP
def c4_like(N, nev, nex, seed):
    return Problem(N=N, nev=nev, nex=nex, spectrum="gap", lo=0.0, hi=10.0, n_low=nev,
                   spacing=0.05, reflectors=8, seed=seed)


def solve_gpu(lib, p, A, tensor=0):
    with lib.Context(lib.default_params(p.N, p.nev, p.nex, fp64_tensor=tensor)) as ctx:
        V = dev(p.start_block(), lib)
        ritz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        resid = torch.zeros_like(ritz)
        ctx.chase_solve(dev(A, lib), V, ritz, resid, lanczos_start=dev(p.lanczos_start(), lib))
    return V, ritz


@pytest.mark.parametrize("N,nev,nex,tensor", [(400, 8, 8, 0), (600, 16, 8, 0), (500, 12, 6, 1)])
def test_eig_vjp_against_oracle(lib, N, nev, nex, tensor):
    p = c4_like(N, nev, nex, N)
    A = p.matrix()
    B = rand_herm(N, N + 3)
    w = uniform01(N, 5, nev) - 0.5
    V, ritz = solve_gpu(lib, p, A, tensor)
    X = V.cpu().numpy()[:, :nev]
    lb, xb = G.c4_loss_adjoints(ritz.cpu().numpy()[:nev], X, w, B)
    with lib.Context(lib.default_params(N, nev, nex, fp64_tensor=tensor)) as ctx:
        Ab = empty_cm(N, N)
        it = ctx.chase_eig_vjp(dev(A, lib), V, ritz, p.ne, nev,
                               torch.from_numpy(lb).cuda(), dev(xb, lib), Ab)
        Ab = Ab.cpu().numpy()
    ref = G.eig_vjp(A, nev, w, G.c4_loss_adjoints(*G.lowest_eigenpairs(A, nev), w, B)[1])
    rel = np.linalg.norm(Ab - ref) / np.linalg.norm(ref)
    print(f"N={N} nev={nev} nex={nex} tensor={tensor}: CG iterations {it}, rel err {rel:.2e}")
    assert rel <= 1e-6


def test_eig_vjp_eigenvalues_only(lib):
    # lam_bar only: Abar = sum_i lam_bar_i x_i x_i^H exactly (Hellmann-Feynman)
    p = c4_like(300, 6, 6, 3)
    A = p.matrix()
    V, ritz = solve_gpu(lib, p, A)
    w = uniform01(3, 9, p.nev)
    with lib.Context(lib.default_params(p.N, p.nev, p.nex)) as ctx:
        Ab = empty_cm(p.N, p.N)
        ctx.chase_eig_vjp(dev(A, lib), V, ritz, p.ne, p.nev, torch.from_numpy(w).cuda(), None, Ab)
        Ab = Ab.cpu().numpy()
    X = V.cpu().numpy()[:, :p.nev]
    want = (X * w[None, :]) @ X.conj().T
    assert np.abs(Ab - want).max() <= 1e-14 * np.abs(want).max() * p.N


def test_eigh_autograd_finite_differences(lib):
    from paper_2309_15595_gb300.autograd import chase_eigh

    p = c4_like(512, 16, 8, 21)
    A0 = p.matrix()
    B = rand_herm(p.N, 22)
    w = uniform01(21, 7, p.nev)
    At = torch.from_numpy(A0).cuda().requires_grad_(True)
    Bt = torch.from_numpy(B).cuda()
    lam, X, _ = chase_eigh(At, torch.from_numpy(p.start_block()).cuda(), p.nev, p.nex,
                           lanczos_start=dev(p.lanczos_start(), lib))
    M = X.conj().T @ Bt @ X
    loss = torch.dot(torch.from_numpy(w).cuda(), lam) + torch.sum(torch.abs(M) ** 2)
    loss.backward()
    Ag = At.grad.cpu().numpy()
    ref = G.eig_vjp(A0, p.nev, w, G.c4_loss_adjoints(*G.lowest_eigenpairs(A0, p.nev), w, B)[1])
    assert np.linalg.norm(Ag - ref) / np.linalg.norm(ref) <= 1e-6

    def L(Am):
        return G.c4_loss(*G.lowest_eigenpairs(Am, p.nev), w, B)

    h = 1e-6
    worst = 0.0
    for k in range(16):  # 16 random Hermitian directions, central differences
        E = rand_herm(p.N, 700 + k)
        E /= np.linalg.norm(E, 2)
        fd = (L(A0 + h * E) - L(A0 - h * E)) / (2 * h)
        an = float(np.real(np.sum(Ag.conj() * E)))
        worst = max(worst, abs(fd - an) / max(abs(an), 1e-3 * abs(L(A0))))
    print(f"worst relative FD mismatch over 16 directions: {worst:.2e}")
    assert worst <= 1e-6
