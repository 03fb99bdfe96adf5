"""Pins of the oracle's heat-equation workload pieces (Sec. 6.1, Sec. 7.2) and
of R_block (Alg. 3): each checked against a closed form, a hand-made case or
an invariant, not against the oracle's own formulas retyped."""
import math
import os
import sys

import numpy as np
import pytest
import scipy.linalg as sla

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_2105_06975_gb300 import workload as W  # noqa: E402
from oracle import covariance as cov, krylov, model as mdl, problem as prb, saddle as sd  # noqa: E402


def small_heat(s=48, N=3, p=12, seed=0, **kw):
    kw.setdefault("msoar_b", (0.4, 0.6, 6))
    kw.setdefault("msoar_q", (0.2, 0.5, 7))
    kw.setdefault("r_blocks", 4)
    kw.setdefault("r_msoar", (1.0, 0.5, 1))
    w = W.HEAT.with_(s=s, N=N, p=p, **kw)
    return w, W.draws(w, seed)


# ------------------------------------------------------------ heat model
def test_heat_model_printed_structure_and_spectrum():
    """Sec. 7.2's M: zero boundary rows and columns, (r, 1-2r, r) inside.  The
    interior block is the Dirichlet second-difference stencil on s-2 points,
    whose eigenvalues are 1 - 4 r sin^2(j pi / (2 (s-1))), j = 1..s-2; the
    boundary adds two zeros.  With r = 0.4 every eigenvalue lies in (-0.6, 1),
    so ||M||_2 < 1 (the hypothesis of Prop. 2)."""
    s, r = 11, 0.4
    M = mdl.heat_model(s, 2, r).dense(1)
    assert np.all(M[0] == 0) and np.all(M[-1] == 0) and np.all(M[:, 0] == 0) and np.all(M[:, -1] == 0)
    for j in range(1, s - 1):
        for k in range(s):
            want = {j - 1: r, j: 1 - 2 * r, j + 1: r}.get(k, 0.0) if 1 <= k <= s - 2 else 0.0
            assert M[j, k] == want
    ev = np.sort(np.linalg.eigvalsh(M))
    j = np.arange(1, s - 1)
    want = np.sort(np.concatenate([[0.0, 0.0], 1 - 4 * r * np.sin(j * np.pi / (2 * (s - 1))) ** 2]))
    assert np.allclose(ev, want, atol=1e-14)
    assert np.linalg.norm(M, 2) < 1.0
    # the same operator for every t, through the banded store
    hm = mdl.heat_model(s, 3, r)
    x = np.random.default_rng(0).standard_normal(s)
    assert np.allclose(hm.apply(3, x), M @ x, atol=1e-15) and np.allclose(hm.apply_T(2, x), M.T @ x, atol=1e-15)


def test_heat_model_is_forward_euler_of_the_heat_equation():
    """One step of M on a sampled Dirichlet eigenfunction sin(pi m x) scales it
    by 1 - 4 r sin^2(pi m dx / 2): forward Euler of u_t = u_xx with
    dt = r dx^2 on the grid x_j = j dx, dx = 1/(s-1)."""
    s, r, m = 41, 0.4, 3
    x = np.arange(s) / (s - 1)
    u = np.sin(np.pi * m * x)
    M = mdl.heat_model(s, 1, r).dense(1)
    lam = 1 - 4 * r * np.sin(np.pi * m / (2 * (s - 1))) ** 2
    assert np.allclose((M @ u)[1:-1], lam * u[1:-1], atol=1e-14)


# ------------------------------------------------------------ modified SOAR
def test_modified_soar_band_geometry_and_shift():
    """The row has 2 maxval + 1 non-zeros; offset i sits at chord 2 sin(i pi /
    (2 maxval)): chord 2 at i = maxval, sqrt(2) at maxval/2, 1 at maxval/3.
    With the shift, lambda_min of the dense matrix is psi exactly (when the
    banded matrix was indefinite)."""
    s, amp, L, mv = 40, 0.4, 0.6, 6
    row = cov.modified_soar_row(s, amp, L, mv)
    assert np.count_nonzero(row) == 2 * mv + 1
    assert np.all(row[mv + 1:s - mv] == 0)
    f = lambda d: amp * (1 + d / L) * math.exp(-d / L)
    assert row[0] == pytest.approx(amp, rel=1e-15)
    assert row[mv] == pytest.approx(f(2.0), rel=1e-14) and row[s - mv] == row[mv]
    assert row[mv // 2] == pytest.approx(f(math.sqrt(2.0)), rel=1e-14)
    assert row[mv // 3] == pytest.approx(f(1.0), rel=1e-14)
    B, delta = cov.modified_soar(s, amp, L, mv, 0.3)
    C = B - delta * np.eye(s)
    assert np.array_equal(C, C.T)
    lam0 = np.linalg.eigvalsh(C)[0]
    assert lam0 < 0 and delta == pytest.approx(-lam0 + 0.3, rel=1e-12)
    assert np.linalg.eigvalsh(B)[0] == pytest.approx(0.3, abs=1e-12)
    # a positive definite band gets no shift
    assert cov.modified_soar_shift(np.array([1.0, 0.1, 0, 0, 0, 0.1]), 0.3) == 0.0
    with pytest.raises(ValueError):
        cov.modified_soar_row(10, amp, L, 5)


def test_modified_soar_band_apply_equals_dense_product():
    s = 37
    row = cov.modified_soar_row(s, 0.2, 0.5, 7)
    delta = cov.modified_soar_shift(row, 0.1)
    V = np.random.default_rng(1).standard_normal((s, 3))
    dense = (cov.circulant(row) + delta * np.eye(s)) @ V
    assert np.allclose(cov.modified_soar_apply(row, delta, V), dense, rtol=1e-13, atol=1e-14)


# ------------------------------------------------------- channel-block R
def test_block_r_generator_structure():
    """Sec. 6.1: R_i = U + U^T symmetric; lambda_min(R_i) = 0.41 exactly
    (Table 2's fixed value); uncorrelated pairs (pcorr = 0) leave zero blocks;
    the other off-diagonal entries lie in [0, pcorr); diagonal blocks are the
    Hadamard product of the sparse factor with the modified SOAR, doubled by
    the symmetrisation."""
    pvec = np.array([5, 4, 4, 3])
    p = int(pvec.sum())
    g = np.random.default_rng(3)
    u = g.random((p, p))
    pcorr = np.array([0.3, 0.0, 0.2, 0.0, 0.4, 0.1])
    R = cov.block_r_matrix(pvec, 0.5, pcorr, u, (1.0, 0.5, 1), 0.41)
    assert np.array_equal(R, R.T)
    assert np.linalg.eigvalsh(R)[0] == pytest.approx(0.41, abs=1e-12)
    pst = np.concatenate([[0], np.cumsum(pvec)])
    S = np.where(u < 0.5, u / 0.5, 0.0)
    shift = R[0, 0] - 2 * S[0, 0] * 1.0            # diagonal: 2 S_jj amp + shift
    q = 0
    for a in range(4):
        for b in range(a + 1, 4):
            blk = R[pst[a]:pst[a + 1], pst[b]:pst[b + 1]]
            if pcorr[q] == 0:
                assert np.all(blk == 0)
            else:
                assert np.all(blk >= 0) and np.all(blk < pcorr[q])
                assert np.allclose(blk, pcorr[q] * S[pst[a]:pst[a + 1], pst[b]:pst[b + 1]], rtol=1e-15)
            q += 1
    for k in range(4):
        sl = slice(pst[k], pst[k + 1])
        m = int(pvec[k])
        Cb = cov.circulant(cov.modified_soar_row(m, 1.0, 0.5, 1))
        D = S[sl, sl] * Cb
        assert np.allclose(R[sl, sl], D + D.T + shift * np.eye(m), rtol=1e-13, atol=1e-14)


# ------------------------------------------------------------ R_block
def blocks_matrix(pvec, consts):
    """Symmetric matrix whose channel block (a, b) is the constant consts[a][b]
    (diagonal blocks dominate so that it is SPD)."""
    pst = np.concatenate([[0], np.cumsum(pvec)])
    p = int(pst[-1])
    R = np.zeros((p, p))
    for a in range(len(pvec)):
        for b in range(len(pvec)):
            R[pst[a]:pst[a + 1], pst[b]:pst[b + 1]] = consts[a][b]
    return R + p * np.eye(p)


def test_r_block_scaled_norms_and_cuts():
    """The scaled Frobenius norm of a constant c block is |c| (||c 1 1^T||_F =
    |c| sqrt(mn)).  A first super-diagonal coupling below tol cuts R there,
    and every coupling across the cut goes with it, higher levels included;
    inside a run of channel blocks every level is kept."""
    pvec = [3, 2, 4, 2]                                  # rows 0-2 | 3-4 | 5-8 | 9-10
    c = [[0, 0.5, 0.2, 0.05], [0.5, 0, 0.6, 0.3], [0.2, 0.6, 0, 0.02], [0.05, 0.3, 0.02, 0]]
    R = blocks_matrix(pvec, c)
    assert cov.block_normvec(R, pvec) == pytest.approx([0.5, 0.6, 0.02], rel=1e-14)
    # tol 0.1: one cut before the last channel block
    assert cov.r_block_cuts(R, pvec, tol=0.1)[0] == [9]
    Rb = cov.r_block(R, pvec, tol=0.1)
    assert np.array_equal(Rb[:9, :9], R[:9, :9])         # includes the level-2 block (c = 0.2)
    assert np.all(R[0:3, 5:9] == 0.2) and np.all(Rb[0:3, 5:9] == 0.2)
    assert np.all(Rb[:9, 9:] == 0) and np.all(Rb[9:, :9] == 0) and np.array_equal(Rb[9:, 9:], R[9:, 9:])
    # tol 0.55: cuts at 3 and 9
    Rb = cov.r_block(R, pvec, tol=0.55)
    assert np.array_equal(Rb, sla.block_diag(R[:3, :3], R[3:9, 3:9], R[9:, 9:]))
    assert np.array_equal(cov.r_block(R, pvec, tol=0.01), R)             # nothing cut
    assert np.array_equal(cov.r_block(R, pvec, tol=np.inf),              # everything cut
                          sla.block_diag(R[:3, :3], R[3:5, 3:5], R[5:9, 5:9], R[9:, 9:]))


def test_r_block_is_exact_for_block_diagonal_r_and_spd():
    """A block-diagonal R (all pcorr = 0) is its own R_block for any tol > 0:
    eig(R_block^{-1} R) = 1.  In general R_block is a direct sum of principal
    submatrices of R, hence SPD, and the runs' eigenvalues interlace."""
    pvec = W.block_sizes(20, 4)
    g = np.random.default_rng(2)
    u = g.random((20, 20))
    R0 = cov.block_r_matrix(pvec, 0.4, np.zeros(6), u, (1.0, 0.5, 1), 0.41)
    Rb = cov.r_block(R0, pvec, tol=1e-3)
    assert np.array_equal(Rb, R0)
    R = cov.block_r_matrix(pvec, 0.4, np.array([0.3, 0.0, 0.2, 0.4, 0.0, 0.1]), u, (1.0, 0.5, 1), 0.41)
    Rb = cov.r_block(R, pvec, tol=0.05)
    lam = np.linalg.eigvalsh(Rb)
    assert lam[0] > 0
    assert lam[0] >= np.linalg.eigvalsh(R)[0] - 1e-12   # Cauchy interlacing on each principal block


def test_r_block_size_and_count_rules():
    """maxsize: the largest run is cut at its row midpoint.  numproc: more runs
    than processors joins the adjacent pair with the smallest total size;
    fewer than numproc - 2 splits the largest run."""
    pvec = [2, 2, 2, 2, 2, 2]
    R = blocks_matrix(pvec, [[0.0 if a == b else 0.5 for b in range(6)] for a in range(6)])
    # all couplings kept: one run of 12 rows; maxsize 8 splits it at 6
    assert cov.r_block_cuts(R, pvec, tol=0.1, maxsize=8)[0] == [6]
    assert cov.r_block_cuts(R, pvec, tol=0.1, maxsize=12)[0] == []
    # all cut: six runs of 2; with 4 processors the first smallest adjacent pair joins
    assert cov.r_block_cuts(R, pvec, tol=1.0, numproc=4)[0] == [4, 6, 8, 10]
    # one run, 5 processors (fewer than numproc - 2 runs): split at the midpoint
    assert cov.r_block_cuts(R, pvec, tol=0.1, numproc=5)[0] == [6]
    # within range: unchanged
    assert cov.r_block_cuts(R, pvec, tol=1.0, numproc=6)[0] == [2, 4, 6, 8, 10]


# ------------------------------------------------------ the heat problem
def test_heat_problem_lu_equals_primal_minimiser_and_krylov():
    """The assembled heat problem (Dirichlet model, modified SOAR B and Q,
    channel-block R) solves to the normal-equations minimiser of the
    linearised cost, and P_I-GMRES with R, R_block and R_diag reaches the LU
    solution."""
    w, dr = small_heat()
    prob, obs, rhs = prb.linear_case(w, dr)
    assert np.linalg.eigvalsh(prob.R)[0] == pytest.approx(0.41, abs=1e-12)
    x_lu = sd.dense_solve(prob, rhs)
    b, d, _ = prob.split(rhs)
    assert np.allclose(b, 0.0)                          # first loop about the background forecast
    x_pr = sd.primal_solve(prob, b.ravel(), d.ravel())
    assert np.linalg.norm(x_lu - x_pr) <= 1e-9 * np.linalg.norm(x_lu)
    pvec = W.block_sizes(w.p, w.r_blocks)
    for rh, blk in [("exact", ()), ("block", (pvec, 0.05, None, None)), ("diag", ())]:
        P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=2, rhat=rh, rblock=blk))
        res = krylov.gmres(prob.A_apply, P.apply, rhs, tol=1e-10)
        assert res.converged
        assert np.linalg.norm(res.x - x_lu) <= 1e-7 * np.linalg.norm(x_lu)


# ------------------------------------------------------------------- L_I
def test_l_i_is_the_printed_matrix_and_a_prefix_sum():
    """Sec. 2.2's L_I: identity blocks on the diagonal, -I below it.  Its
    inverse is block lower triangular with every block I, so L_I^{-1} v is the
    running sum over time levels and L_I^{-T} v the sum from the end.  Inside
    the preconditioner it replaces only L-hat: the saddle matrix keeps M."""
    s, N = 5, 4
    im = mdl.IdentityModel(s, N)
    Ld = mdl.L_dense(im)
    want = np.eye((N + 1) * s) - np.eye((N + 1) * s, k=-s)
    assert np.array_equal(Ld, want)
    v = np.random.default_rng(4).standard_normal((N + 1, s))
    assert np.allclose(mdl.LM_inv(im, v, N + 1), np.cumsum(v, axis=0), atol=1e-15)
    assert np.allclose(mdl.LM_inv_T(im, v, N + 1), np.cumsum(v[::-1], axis=0)[::-1], atol=1e-15)
    w, dr = small_heat(s=24, N=3, p=6)
    prob = prb.linear_problem(w, dr)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=prob.N + 1, lhat_identity=True))
    ns = prob.s * (prob.N + 1)
    assert np.array_equal(P.dense()[:ns, -ns:], mdl.L_dense(mdl.IdentityModel(prob.s, prob.N)))
    assert np.array_equal(prob.A_dense()[:ns, -ns:], mdl.L_dense(prob.model))


def test_r_block_one_cut_spectrum_pairs_about_one():
    """With one cut, R = R_block + E with E zero on the two diagonal runs, so
    R_block^{-1/2} E R_block^{-1/2} has eigenvalues in +- pairs and eig(R_block^{-1}
    R) = 1 +- mu: lambda_min + lambda_max = 2.  Table 2's R_block columns show
    that pairing in every row (to the printed 4 digits), and the oracle's
    R_block on a channel-block R_i with one cut has it exactly.  The same
    table fixes lambda_min(R_i) = 0.41 in every row."""
    rows = [list(map(float, ln.split())) for ln in open(os.path.join(ROOT, "tests", "golden", "table2_eigs.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 6
    for p, rmin, rmax, dmin, dmax, bmin, bmax, *_ in rows:
        assert bmin + bmax == pytest.approx(2.0, abs=2e-4)
        assert rmin == 0.41
    pvec = W.block_sizes(40, 4)
    u = np.random.default_rng(9).random((40, 40))
    R = cov.block_r_matrix(pvec, 0.4, np.array([0.3, 0.2, 0.1, 0.4, 0.25, 0.35]), u, (1.0, 0.5, 2), 0.41)
    nv = cov.block_normvec(R, pvec)
    tol = 0.5 * (np.sort(nv)[0] + np.sort(nv)[1])      # exactly one first super-diagonal coupling below tol
    cuts, _ = cov.r_block_cuts(R, pvec, tol)
    assert len(cuts) == 1
    ev = np.sort(sla.eigh(R, cov.r_block(R, pvec, tol), eigvals_only=True))
    assert ev[0] + ev[-1] == pytest.approx(2.0, abs=1e-10)
    assert np.allclose(ev + ev[::-1], 2.0, atol=1e-10)


def test_band_covariance_problem_equals_dense_problem():
    """The heat window with B and Q applied through their modified SOAR bands
    (oracle.saddle.BandCovProblem, for sizes where dense B, Q do not fit) gives
    the dense problem's A v and P_I^{-1} v on a window where both fit."""
    w = W.small(W.HEAT, s=300, N=3, p=60)
    dr = W.draws(w, 2)
    prob, obs, rhs = prb.linear_case(w, dr)
    bp = prb.heat_band_problem(w, dr)
    assert np.array_equal(bp.R, prob.R)
    v = W.random_vector(prob.n, 4)
    assert np.linalg.norm(bp.A_apply(v) - prob.A_apply(v)) <= 1e-14 * np.linalg.norm(prob.A_apply(v))
    o = sd.PrecondOptions(kind="PI", k=2)
    a, b = sd.Preconditioner(bp, o).apply(v), sd.Preconditioner(prob, o).apply(v)
    assert np.linalg.norm(a - b) <= 1e-13 * np.linalg.norm(b)
