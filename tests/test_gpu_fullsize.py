"""The tensor-core paths at the sizes the benchmark runs them, against the oracle.

* The FP64-accurate digit-sliced filter (fp64_tensor = 1) and the split-BF16 x3
  filter over all 1300 columns of the N = 20000 workload at degree 20, with
  the grouped raster order of both kernels engaged (it starts above 1024 and
  2048 rows), checked on sampled columns against the oracle's filter (columns
  are independent in the filter).
* The digit-sliced product at the longest inner dimension the workloads use,
  K = 2N = 80000 (N = 40000), through a degree-2 filter step and the residual
  norms on a few columns, against the oracle with the same A copied to the host.
* The Rayleigh-Ritz eigensolver at order n = 1300 on a clustered spectrum
  (clusters of four with spacing 1e-3), where the FP32 Jacobi sweeps cannot
  separate the pairs and the FP64 finish runs.

Error bounds. Digit-sliced product: the truncation errors of the K terms add
with random signs to about sqrt(K) 2^-48 of max|a| max|y| per entry (six
digits, levels 2-5 exact, 6-7 in FP32 per 256-long chunk). The bound per
filter column is degs * 2^-42 * sqrt(K / 1400) of the column's largest entry,
the N <= 700 bound of the small-size tests scaled by the sqrt(K) growth of the
truncation error. Split-BF16 x3: degs * 2^-15 of the column's largest entry. The
split products carry about 2^-16 per step (a CPU emulation of them gives 1.1e-5
per degree on this geometric spectrum; measured here 1.75e-5 per degree with
the FP32 state and accumulation, so the bound leaves a factor 1.7); the tensor
cores' FP32 accumulation enters only per 256-long K chunk, so neither the error
nor the bound grows with N (before the chunked accumulation the same test
measured 1e-2). Measured values are printed.
"""
import numpy as np
import pytest

from oracle import chase_oracle as O
from synth import Problem, complex_normal, config_problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def host_matrix(Ad):
    """Copy of a column-major device matrix to a Fortran-ordered host array in
    column slabs (no full-size temporary on either side)."""
    N = Ad.shape[0]
    A = np.empty((N, N), dtype=np.complex128, order="F")
    slab = max(1, (1 << 30) // (16 * N))
    for j in range(0, N, slab):
        A[:, j:j + slab] = Ad[:, j:j + slab].cpu().numpy()
    return A


def spectral(p):
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    return (b_sup + lam[p.ne - 1]) / 2, (b_sup - lam[p.ne - 1]) / 2, lam[0]


def test_digit_sliced_product_at_k80000(lib):
    """N = 40000 (K = 80000), four columns: one degree-2 filter step and the
    residual norms with the tensor-core FP64 products, against the oracle."""
    p = config_problem("C3")
    N = p.N
    Ad = p.matrix_torch("cuda")
    A = host_matrix(Ad)
    ncols = 4
    V0 = np.asfortranarray(complex_normal(3, 95, N * ncols).reshape(ncols, N).T)
    lam = p.eigenvalues()
    b_sup = lam[-1] * 1.01
    c, e, mu1 = (b_sup + lam[2999]) / 2, (b_sup - lam[2999]) / 2, lam[0]
    degs = np.full(ncols, 2, dtype=np.int32)
    theta = np.linspace(lam[0], lam[100], ncols)
    with lib.Context(lib.default_params(N, ncols, 0, fp64_tensor=1)) as ctx:
        Vd = lib.colmajor(torch.from_numpy(V0).cuda())
        ctx.chase_filter(Ad, Vd, ncols, degs, c, e, mu1)
        Y = Vd.cpu().numpy()
        Wd = lib.colmajor(torch.from_numpy(V0).cuda())
        r = torch.zeros(ncols, dtype=torch.float64, device="cuda")
        ctx.chase_residuals(Ad, Wd, torch.from_numpy(theta).cuda(), ncols, r)
        r = r.cpu().numpy()
    del Ad
    torch.cuda.empty_cache()
    ref = O.chebyshev_filter(A, V0, degs, c, e, mu1)
    rel = np.abs(Y - ref).max(axis=0) / np.abs(ref).max(axis=0)
    bound = degs * 2.0 ** -42 * np.sqrt(2 * N / 1400)
    rr = O.residuals(A, V0, theta)
    rres = np.abs(r - rr) / rr
    print(f"K=80000: filter rel err {rel}, bound {bound[0]:.2e}; residual rel err {rres}")
    assert np.all(rel <= bound)
    assert np.all(rres <= 1e-9)


@pytest.fixture(scope="module")
def c2():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    p = config_problem("C2")
    Ad = p.matrix_torch("cuda")
    return p, Ad, host_matrix(Ad)


@pytest.mark.parametrize("mode", ["fp64_tensor", "mixed"])
def test_filter_full_size_sampled(lib, c2, mode):
    p, Ad, A = c2
    N, ne = p.N, p.ne
    V0 = p.start_block()
    c, e, mu1 = spectral(p)
    degs = np.full(ne, 20, dtype=np.int32)
    cols = np.array([0, 129, 700, ne - 1])
    if mode == "fp64_tensor":
        prm = lib.default_params(N, p.nev, p.nex, fp64_tensor=1)
        prec = lib.CHASE_FP64
    else:
        prm = lib.default_params(N, p.nev, p.nex, precision=lib.CHASE_MIXED_BF16X3)
        prec = lib.CHASE_MIXED_BF16X3
    with lib.Context(prm) as ctx:
        Vd = lib.colmajor(torch.from_numpy(V0).cuda())
        ctx.chase_filter(Ad, Vd, ne, degs, c, e, mu1, precision=prec)
        Y = Vd[:, torch.from_numpy(cols).cuda()].cpu().numpy()
    ref = O.chebyshev_filter(A, V0[:, cols], degs[cols], c, e, mu1)
    rel = np.abs(Y - ref).max(axis=0) / np.abs(ref).max(axis=0)
    if mode == "fp64_tensor":
        bound = degs[cols] * 2.0 ** -42 * np.sqrt(2 * N / 1400)
    else:
        bound = degs[cols] * 2.0 ** -15
    print(f"{mode} N={N} ncols={ne} deg 20: rel err per sampled column {rel}, bound {bound[0]:.2e}")
    assert np.all(np.isfinite(Y))
    assert np.all(rel <= bound)


def clustered_rr_input(N, n, seed):
    """A (N x N) with the clustered low spectrum of the N = 40000 workload and Q
    an orthonormal basis of its n lowest eigenvectors mixed by a unitary W, so
    that Q^H A Q has exactly those n eigenvalues (clusters of four, spacing
    1e-3)."""
    p = Problem(N=N, nev=n - n // 4, nex=n // 4, spectrum="clusters", lo=-2.0, hi=50.0,
                n_low=n, spacing=1e-3, reflectors=8, seed=seed)
    A = p.matrix()
    X = p.eigenvectors(np.arange(n))
    W = np.linalg.qr(complex_normal(seed, 94, n * n).reshape(n, n))[0]
    return p, A, np.asfortranarray(X @ W)


@pytest.mark.parametrize("tensor", [0, 1])
def test_rayleigh_ritz_clustered_n1300(lib, tensor):
    N, n = 3000, 1300
    p, A, Q = clustered_rr_input(N, n, 31)
    th_o, V_o = O.rayleigh_ritz(A, Q)
    lam = p.eigenvalues()[:n]
    nA = p.norm2()
    with lib.Context(lib.default_params(N, p.nev, p.nex, fp64_tensor=tensor)) as ctx:
        Vd = lib.colmajor(torch.from_numpy(Q).cuda())
        ritz = torch.zeros(n, dtype=torch.float64, device="cuda")
        ctx.chase_rayleigh_ritz(lib.colmajor(torch.from_numpy(A).cuda()), Vd, n, ritz)
        th = ritz.cpu().numpy()
        V = Vd.cpu().numpy()
    err_o = np.abs(th - th_o).max() / nA
    err_x = np.abs(th - lam).max() / nA
    orth = np.abs(V.conj().T @ V - np.eye(n)).max()
    res = (np.linalg.norm(A @ V - V * th[None, :], axis=0) / nA).max()
    print(f"RR n={n} clustered (tensor={tensor}): |dtheta| vs oracle {err_o:.2e}, vs exact "
          f"{err_x:.2e}, orth {orth:.2e}, max rel resid {res:.2e}")
    assert np.all(np.diff(th) >= 0)
    assert err_o <= 1e-12 and err_x <= 1e-12
    assert orth <= 1e-12
    assert res <= 1e-11
    # each cluster's invariant subspace against the oracle's: sine of the largest
    # principal angle as the norm of the part of V's cluster block outside the
    # oracle's (accurate at small angles, unlike sqrt(1 - cos^2))
    starts = np.r_[0, np.nonzero(np.diff(th_o) > 5e-4)[0] + 1, n]
    worst = 0.0
    for a, b in zip(starts[:-1], starts[1:]):
        Vo, Vg = V_o[:, a:b], V[:, a:b]
        worst = max(worst, float(np.linalg.norm(Vg - Vo @ (Vo.conj().T @ Vg), 2)))
    print(f"  worst cluster subspace angle {worst:.2e}")
    assert worst <= 1e-8


def test_solve_clustered_uses_cluster_finish(lib):
    """A C3-like solve (clusters of four, spacing 1e-3): the eigensolver's FP64
    finish runs per cluster (no full FP64 sweep is needed on the clustered
    Rayleigh-Ritz matrices) and the solve reaches the exact spectrum."""
    p = config_problem("C3", N=2000, nev=225, nex=75, n_low=300)
    A = p.matrix()
    with lib.Context(lib.default_params(p.N, p.nev, p.nex, max_iter=40)) as ctx:
        Vd = lib.colmajor(torch.from_numpy(p.start_block()).cuda())
        ritz = torch.zeros(p.ne, dtype=torch.float64, device="cuda")
        resid = torch.zeros_like(ritz)
        st = ctx.chase_solve(lib.colmajor(torch.from_numpy(A).cuda()), Vd, ritz, resid,
                             lanczos_start=lib.colmajor(torch.from_numpy(p.lanczos_start()).cuda()))
        got = ritz.cpu().numpy()[:p.nev]
        V = Vd.cpu().numpy()[:, :p.nev]
    nA = p.norm2()
    print(f"clustered solve: iters {st['iters']}, cluster finishes {st['heev_cluster_solves']}, "
          f"largest cluster {st['heev_cluster_max']}, FP64 sweeps {st['heev_fp64_sweeps']}")
    assert st["status"] == 0
    assert np.abs(got - p.eigenvalues()[:p.nev]).max() <= 1e-10 * nA
    assert (np.linalg.norm(A @ V - V * got[None, :], axis=0) / nA).max() <= 1e-10
    assert np.abs(V.conj().T @ V - np.eye(p.nev)).max() <= 1e-12


def test_qr_localized_block_at_k80000(lib):
    """CholeskyQR2 with the tensor-core products of X = Q0 T at N = 40000
    (K = 80000 in the Grams), Q0 orthonormal with one entry near 1 per column.
    The Grams' diagonals add squared digits coherently over K; summed across the
    256-long chunks in FP32 they were off by about 2^-44 of the scale at this K,
    which left orthogonality near 1e-12 here (2e-11 in the C3 solve); with the
    FP64 sums it stays at the digit rounding, a few 1e-14."""
    N, n = 40000, 128
    rng = np.random.default_rng(40)
    E = np.zeros((N, n), dtype=np.complex128)
    E[rng.permutation(N)[:n], np.arange(n)] = 1.0
    Z = complex_normal(40, 98, N * n).reshape(n, N).T
    Q0, R0 = np.linalg.qr(E + 0.02 * Z)
    Q0 = Q0 * (np.diag(R0) / np.abs(np.diag(R0)))[None, :]
    T = np.eye(n) + np.triu(complex_normal(41, 99, n * n).reshape(n, n), 1) * (0.3 / np.sqrt(n))
    X = np.asfortranarray(Q0 @ T)
    with lib.Context(lib.default_params(N, n, 0, fp64_tensor=1)) as ctx:
        Xd = lib.colmajor(torch.from_numpy(X).cuda())
        v = ctx.chase_qr(Xd, n, 100.0)
        G = (Xd.mH @ Xd).cpu().numpy()
        Q = Xd.cpu().numpy()
    orth = np.abs(G - np.eye(n)).max()
    fwd = np.abs(Q - Q0).max()
    print(f"localized QR N={N} n={n}: variant {v}, orth {orth:.2e}, |Q - Q0| {fwd:.2e}")
    assert v == lib.CHASE_QR_CHOLQR2
    assert orth <= 1e-13
    assert fwd <= 1e-12
