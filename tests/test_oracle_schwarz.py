"""Pins of the oracle's one-level Schwarz preconditioners and ILU(k) (Section 3.1)."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import torch

from oracle import discretization as disc
from oracle import schwarz
from paper_2007_13966_gb300 import synthetic as syn


def jac(nx, ny, nz, seed=4):
    res = syn.small_3d(nx, ny, nz, seed=seed)
    prob = disc.Problem(res)
    p = syn.random_pressure(res, seed)
    _, J = disc.residual(prob, p, 0.98 * p, 0.97 * p, 8640.0, 2, want_jac=True)
    return disc.jacobian_csr(res.grid, J), (nx, ny, nz)


def test_split_axis_remainder_first_and_cover():
    for n in (1, 7, 16, 61):
        for P in (1, 2, 3, 4):
            if P > n:
                continue
            s = schwarz.split_axis(n, P)
            sizes = np.diff(s)
            assert s[0] == 0 and s[-1] == n
            assert sizes.max() - sizes.min() <= 1
            assert list(sizes) == sorted(sizes, reverse=True)


def test_partition_owned_cells_cover_once():
    dims = (13, 9, 7)
    boxes = schwarz.partition(dims, (3, 2, 2), 2)
    cnt = np.zeros(np.prod(dims), dtype=int)
    for b in boxes:
        np.add.at(cnt, b.idx[b.own], 1)
        # overlapped box = owned box grown by delta, clipped at the boundary
        for a in range(3):
            assert b.e0[a] == max(b.o0[a] - 2, 0)
            assert b.e1[a] == min(b.o1[a] + 2, dims[a])
    assert np.all(cnt == 1)


def test_ilu0_on_stencil_changes_only_the_diagonal():
    A, dims = jac(5, 4, 3)
    L, U = schwarz.ilu_numeric(A, schwarz.iluk_symbolic(A, 0))
    pattern = (abs(A) > 0).astype(int)
    LU_pat = ((abs(L) + abs(U)) > 0).astype(int)
    assert (pattern != LU_pat).nnz == 0
    d = schwarz.ilu0_stencil_pivots(A)
    assert np.allclose(U.diagonal(), d, rtol=1e-13, atol=0)
    # U's off-diagonals are A's; L_nm = a_nm / d_m
    Aoff_up = sp.triu(A, 1).tocsr()
    assert abs(sp.triu(U, 1) - Aoff_up).max() == 0
    Alow = sp.tril(A, -1).tocoo()
    Ld = L.todok()
    for i, j, v in zip(Alow.row, Alow.col, Alow.data):
        assert abs(Ld[i, j] - v / d[j]) <= 1e-14 * abs(v / d[j])


def test_ilu0_tridiagonal_is_exact_lu():
    A, _ = jac(12, 1, 1)
    L, U = schwarz.ilu_numeric(A, schwarz.iluk_symbolic(A, 0))
    LU = (L + sp.eye(A.shape[0])) @ U
    assert abs(LU - A).max() <= 1e-13 * abs(A).max()


def test_iluk_large_k_is_exact_lu():
    A, _ = jac(4, 4, 2)
    L, U = schwarz.ilu_numeric(A, schwarz.iluk_symbolic(A, 40))
    LU = ((L + sp.eye(A.shape[0])) @ U).toarray()
    assert np.abs(LU - A.toarray()).max() <= 1e-12 * abs(A).max()


def test_iluk_fill_grows_with_k():
    A, _ = jac(6, 5, 3)
    nnz = [sum(len(r) for r in schwarz.iluk_symbolic(A, k)) for k in (0, 1, 2)]
    assert nnz[0] == A.nnz and nnz[0] < nnz[1] < nnz[2]


def test_one_subdomain_left_ras_is_global_ilu0():
    A, dims = jac(6, 5, 4)
    M = schwarz.Schwarz(A, dims, (1, 1, 1), 2, schwarz.LEFT_RAS)
    L, U = schwarz.ilu_numeric(A, schwarz.iluk_symbolic(A, 0))
    r = syn.random_vector(A.shape[0], 3)
    y = sp.linalg.spsolve_triangular((L + sp.eye(A.shape[0])).tocsr(), r, lower=True)
    z = sp.linalg.spsolve_triangular(U.tocsr(), y, lower=False)
    assert np.allclose(M(r), z, rtol=1e-13, atol=1e-13 * np.abs(z).max())


def test_zero_overlap_all_variants_are_block_jacobi():
    A, dims = jac(6, 6, 2)
    parts = (2, 3, 1)
    Ms = [schwarz.Schwarz(A, dims, parts, 0, k, sub="lu") for k in
          (schwarz.AS, schwarz.LEFT_RAS, schwarz.RIGHT_RAS)]
    Ad = A.toarray()
    BJ = np.zeros_like(Ad)
    for b in schwarz.partition(dims, parts, 0):
        ix = np.ix_(b.idx, b.idx)
        BJ[ix] = np.linalg.inv(Ad[ix])
    for M in Ms:
        assert np.abs(M.dense() - BJ).max() <= 1e-12 * np.abs(BJ).max()


def test_full_overlap_lu_ras_is_exact_inverse():
    A, dims = jac(6, 4, 3)
    M = schwarz.Schwarz(A, dims, (2, 2, 1), 10, schwarz.LEFT_RAS, sub="lu")
    Ainv = np.linalg.inv(A.toarray())
    assert np.abs(M.dense() - Ainv).max() <= 1e-10 * np.abs(Ainv).max()


def test_left_ras_transpose_is_right_ras_of_transpose():
    A, dims = jac(6, 5, 2)
    parts = (2, 2, 1)
    ML = schwarz.Schwarz(A, dims, parts, 1, schwarz.LEFT_RAS, sub="lu").dense()
    MR = schwarz.Schwarz(A.T.tocsr(), dims, parts, 1, schwarz.RIGHT_RAS, sub="lu").dense()
    assert np.abs(ML.T - MR).max() <= 1e-12 * np.abs(ML).max()


def test_as_is_sum_over_overlapped_subdomains():
    A, dims = jac(5, 5, 1)
    parts = (2, 2, 1)
    M = schwarz.Schwarz(A, dims, parts, 1, schwarz.AS, sub="lu").dense()
    Ad = A.toarray()
    ref = np.zeros_like(Ad)
    for b in schwarz.partition(dims, parts, 1):
        ix = np.ix_(b.idx, b.idx)
        ref[ix] += np.linalg.inv(Ad[ix])
    assert np.abs(M - ref).max() <= 1e-12 * np.abs(ref).max()


def test_bf16_rounding_matches_torch():
    x = np.random.default_rng(0).standard_normal(10000).astype(np.float32) * 1e3
    ours = schwarz.round_bf16(x)
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    assert np.array_equal(ours, ref)


@pytest.mark.parametrize("prec", [32, 16])
def test_reduced_precision_factors_close_to_fp64(prec):
    A, dims = jac(6, 5, 4)
    r = syn.random_vector(A.shape[0], 9)
    z64 = schwarz.Schwarz(A, dims, (2, 2, 2), 1)(r)
    zlo = schwarz.Schwarz(A, dims, (2, 2, 2), 1, prec=prec)(r)
    err = np.abs(zlo - z64).max() / np.abs(z64).max()
    assert err < (1e-5 if prec == 32 else 3e-2)
    assert err > 0


def test_restricted_variants_beat_classical_as_table_5():
    """Table 5's orderings as a trend check (FGMRES(30) to 1e-6, 4 x 4 subdomains):
    at every overlap 1 to 3 left- and right-RAS need fewer iterations than
    classical AS, and a wider overlap does not make RAS worse than overlap 1."""
    from oracle import krylov
    A, dims = jac(32, 32, 1, seed=2)
    b = syn.random_vector(A.shape[0], 4)
    its = {}
    for kind in (schwarz.AS, schwarz.LEFT_RAS, schwarz.RIGHT_RAS):
        for d in (1, 2, 3):
            M = schwarz.Schwarz(A, dims, (4, 4, 1), d, kind=kind)
            _, info = krylov.fgmres(lambda v: A @ v, M, b, rtol=1e-6, restart=30, maxit=3000)
            its[kind, d] = info["iters"]
    for d in (1, 2, 3):
        assert its[schwarz.LEFT_RAS, d] < its[schwarz.AS, d], its
        assert its[schwarz.RIGHT_RAS, d] < its[schwarz.AS, d], its
    for kind in (schwarz.LEFT_RAS, schwarz.RIGHT_RAS):
        assert max(its[kind, 2], its[kind, 3]) <= its[kind, 1], its


@pytest.mark.parametrize("dims,parts,seed", [((32, 32, 1), (4, 4, 1), 2), ((16, 16, 8), (2, 2, 2), 3)])
def test_more_fill_fewer_iterations_table_3(dims, parts, seed):
    """Table 3's ordering as a trend check (classical AS, overlap 1, FGMRES(30) to
    1e-6): ILU(0) > ILU(1) > ILU(2) > ILU(4) > exact LU in iterations, in 2D and 3D."""
    from oracle import krylov
    A, dims = jac(*dims, seed=seed)
    b = syn.random_vector(A.shape[0], 4)
    its = []
    for sub, k in (("ilu", 0), ("ilu", 1), ("ilu", 2), ("ilu", 4), ("lu", 0)):
        M = schwarz.Schwarz(A, dims, parts, 1, kind=schwarz.AS, sub=sub, ilu_k=k)
        _, info = krylov.fgmres(lambda v: A @ v, M, b, rtol=1e-6, restart=30, maxit=3000)
        its.append(info["iters"])
    assert all(a > b_ for a, b_ in zip(its, its[1:])), its
