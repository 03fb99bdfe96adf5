"""OZAKI mode (not in the paper): the covariance / factor products with two or
more right-hand sides on the tensor cores, by exact BF16 digit products
(7 balanced base-128 digits per operand below a power-of-two scale per row /
column, the 28 products of significance levels 0..6 accumulated exactly in
FP32, combined in double-float).  One-column products run in double-float.

Parity with the FP64 oracle on the same seeded inputs:
  * A v within 1e-11 (2-norm, relative) -- each operand keeps 47 bits below
    its row / column scale and a product's error is ~2^-44 K max|a_i.| max|x_.c|,
    close to the DF32 mode's ~48-bit products;
  * P^{-1} v within 1e-9 (as DF32 mode);
  * the solve meets the true FP64 residual with the oracle's operator, in the
    same number of iterations as DF32 mode (+-2, 5 %).
Shapes cover ragged tiles: rows and k not multiples of 128 / 16, one-column
time levels, column tiles of 2..64 columns and a 65th column, k-ranges longer
than one exact segment (512).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2105_06975_gb300 import workload as W

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - collected on CPU machines too
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2105_06975_gb300 import wc4d as L  # noqa: E402
from oracle import problem as prb, saddle as sd  # noqa: E402

DEV = "cuda"


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(DEV)


def case(s, N, p, obs="random", seed=0):
    w = W.small(W.TINY, s=s, N=N, p=p).with_(obs=obs)
    return w, W.draws(w, seed)


def popts(kind, k):
    return sd.PrecondOptions(kind=kind, k=k, rhat="exact", shat="paper", dhat="exact", kappa_max=100.0)


@pytest.mark.parametrize("s,N,p", [
    (203, 6, 77),     # rows / k ragged; Q: one 6-column tile; R: 7 columns
    (256, 64, 128),   # Q: one full 64-column tile; R: 64 + a one-column remainder
    (300, 70, 130),   # Q: 64 + 6 columns; R: 64 + 7
    (130, 1, 40),     # Q: one column (double-float only); R: a 2-column tile
    (600, 3, 520),    # k = 600 and 520: several exact segments per tile
])
def test_ozaki_products_match_oracle_and_df32(s, N, p):
    w, dr = case(s, N, p, seed=3)
    prob = prb.linear_problem(w, dr)
    k = min(3, N + 1)
    o = L.make_opts(precond="PI", k=k, precision="ozaki")
    Z = L.Problem.from_workload(w, dr, o)
    D = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=k, precision="df32"))
    v = W.random_vector(prob.n, 11)
    az = Z.apply_saddle(to_dev(v)).cpu().numpy()
    assert np.all(np.isfinite(az))
    assert rel(az, prob.A_apply(v)) < 1e-11
    assert rel(az, D.apply_saddle(to_dev(v)).cpu().numpy()) < 1e-11
    P = sd.Preconditioner(prob, popts("PI", k))
    pz = Z.apply_precond("PI", to_dev(v)).cpu().numpy()
    assert rel(pz, P.apply(v)) < 1e-9
    # a zero vector gives exactly zero
    zero = Z.apply_saddle(torch.zeros(prob.n, dtype=torch.float64, device=DEV))
    assert float(zero.abs().max()) == 0.0
    Z.close()
    D.close()


def test_ozaki_column_maxima_next_to_a_power_of_two():
    """A column whose largest magnitude lies just below its power-of-two scale
    is the edge of the digit split (the balanced digits of a 47-bit integer
    fill all seven 7-bit fields); signs, exact zeros and entries 2^-60 below
    the maximum ride along."""
    w, dr = case(203, 6, 77, seed=5)
    prob = prb.linear_problem(w, dr)
    Z = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=3, precision="ozaki"))
    v = W.random_vector(prob.n, 21)
    s, N, p = w.s, w.N, w.p
    ns = s * (N + 1)
    rng = np.random.default_rng(7)
    for off, m in ((0, s), (ns, p)):
        blk = v[off:off + m * (N + 1)].reshape(N + 1, m)   # one time level per row of blk (a view)
        for c in range(N + 1):
            col = blk[c]
            j = int(np.argmax(np.abs(col)))
            col *= (1.0 - 2.0 ** -45) * 2.0 ** (c - 3) / abs(col[j])
            col[j] = (-1.0 if c % 2 else 1.0) * abs(col[j])
            col[rng.integers(0, m, 3)] = 0.0
            col[(j + 1) % m] = 2.0 ** -60
    az = Z.apply_saddle(to_dev(v)).cpu().numpy()
    assert rel(az, prob.A_apply(v)) < 1e-11
    P = sd.Preconditioner(prob, popts("PI", 3))
    assert rel(Z.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    Z.close()


@pytest.mark.parametrize("s,N,p,gemv_ops,tiles", [
    (256, 64, 128, 1, 1),   # B on one column; Q's 64 columns from its shared digit tiles
    (203, 6, 77, 1, 0),     # rows and k ragged: Q's padded tiles are not shared
    (130, 1, 40, 2, 0),     # N = 1: B and Q both on one column
])
def test_toeplitz_products(s, N, p, gemv_ops, tiles):
    """The library's SOAR B and Q of the periodic grid are symmetric Toeplitz
    (entry (i, k) a function of |i - k| only, Sec. 6.1).  Under toeplitz_gemv
    AUTO (the default) their one-column products read the split first row,
    and Q's tensor-core products read one digit tile per offset 128 R - 16 K
    when every tile equals it (not with padded tiles); both must give bitwise
    the products of the dense operator (OFF), A v and P_I^-1 v alike.  The
    launch's FP64 byte floor counts the first row instead of the s^2 entries
    of each such operator, and its digit-form bytes each shared tile once.  A
    B and Q perturbed off the Toeplitz structure (one interior entry pair,
    1e-12 relative) keep the dense path under AUTO."""
    w, dr = case(s, N, p, seed=5)
    prob = prb.linear_problem(w, dr)
    k = min(3, N + 1)
    v = to_dev(W.random_vector(prob.n, 21))

    def run(mode, **dense):
        o = L.make_opts(precond="PI", k=k, precision="ozaki", toeplitz_gemv=mode)
        G = L.Problem.from_workload(w, dr, o, dense=bool(dense), **dense)
        L.wc4d_set_profiling(True)
        try:
            L.wc4d_reset_stats()
            az = G.apply_saddle(v).cpu().numpy()
            st = L.wc4d_get_stats()
            pz = G.apply_precond("PI", v).cpu().numpy()
        finally:
            L.wc4d_set_profiling(False)
            G.close()
        assert st.gemmtc_launches == 1
        return az, pz, st.gemmtc_alg_bytes, st.gemmtc_bytes

    az1, pz1, alg1, by1 = run(L.WC4D_TOEPLITZ_AUTO)
    az0, pz0, alg0, by0 = run(L.WC4D_TOEPLITZ_OFF)
    assert np.all(np.isfinite(az1))
    assert np.array_equal(az1, az0) and np.array_equal(pz1, pz0)
    assert alg0 - alg1 == (gemv_ops + tiles) * 8.0 * (s * s - s)
    rt, nkb = -(-s // 128), -(-s // 16)
    shared = tiles * (rt * nkb - min(rt * nkb, nkb + 8 * (rt - 1))) * 7 * 128 * 16 * 2
    assert by0 - by1 == gemv_ops * 8.0 * (s * s - s) + shared
    assert rel(az1, prob.A_apply(v.cpu().numpy())) < 1e-11
    Bp, Qp = prob.B.copy(), prob.Q.copy()
    for M in (Bp, Qp):
        M[1, 2] *= 1.0 + 1e-12
        M[2, 1] = M[1, 2]
    dense = dict(B=Bp, Q=Qp, R=prob.R)
    azp1, pzp1, algp1, byp1 = run(L.WC4D_TOEPLITZ_AUTO, **dense)
    azp0, pzp0, algp0, byp0 = run(L.WC4D_TOEPLITZ_OFF, **dense)
    assert np.array_equal(azp1, azp0) and np.array_equal(pzp1, pzp0)
    assert algp1 == algp0 == alg0 and byp1 == byp0 == by0


def test_ozaki_block_diagonal_preconditioner():
    w, dr = case(203, 6, 77, seed=2)
    prob = prb.linear_problem(w, dr)
    Z = L.Problem.from_workload(w, dr, L.make_opts(precond="PD", k=3, precision="ozaki"))
    v = W.random_vector(prob.n, 8)
    P = sd.Preconditioner(prob, popts("PD", 3))
    assert rel(Z.apply_precond("PD", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-9
    Z.close()


@pytest.mark.parametrize("kind,krylov", [("PI", "gmres"), ("PD", "gmres"), ("PD", "minres")])
def test_ozaki_solve_matches_df32_and_lu(kind, krylov):
    w, dr = case(203, 6, 77, seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    res = {}
    for prec in ("df32", "ozaki"):
        o = L.make_opts(precond=kind, k=3, precision=prec, krylov=krylov, tol=1e-10, maxit=1500)
        G = L.Problem.from_workload(w, dr, o)
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, (prec, info.as_dict())
        xg = x.cpu().numpy()
        r = rhs - prob.A_apply(xg)
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-10
        assert rel(xg, x_lu) < 1e-6
        res[prec] = info.iters
        G.close()
    assert abs(res["ozaki"] - res["df32"]) <= 2 + 0.05 * res["df32"], res


def test_ozaki_nonfinite_input_is_reported():
    w, dr = case(203, 6, 77, seed=2)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=3, precision="ozaki", maxit=50))
    bad = rhs.copy()
    bad[5] = np.nan
    v = W.random_vector(prob.n, 4)
    v[prob.n // 2] = np.inf
    av = G.apply_saddle(to_dev(v)).cpu().numpy()
    assert not np.all(np.isfinite(av))
    with pytest.raises(L.WC4DError) as e:
        G.solve(to_dev(bad))
    assert e.value.code == L.WC4D_ERR_NONFINITE
    # the problem stays usable
    x, info = G.solve(to_dev(rhs))
    assert info.status in (0, L.WC4D_ERR_MAXIT)
    G.close()


@pytest.mark.slow
def test_ozaki_scale_workload():
    """s=2048, N=64, p=1024 (n = 332,800): the benchmark's launch configuration.
    A v within 1e-11 of the oracle, P_I^{-1} v within 1e-7 (the bound of the
    FP64 mode at this size: kappa(R) = 2.6e9), and the solve meets the 1e-6
    relative residual with the oracle's operator."""
    w = W.SCALE
    dr = W.draws(w, 0)
    prob, obs, rhs = prb.linear_case(w, dr)
    v = W.random_vector(prob.n, 3)
    P = sd.Preconditioner(prob, popts("PI", 4))
    o = L.make_opts(precond="PI", k=4, precision="ozaki", tol=1e-6, maxit=1000)
    G = L.Problem.from_workload(w, dr, o)
    assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
    assert rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), P.apply(v)) < 1e-7
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0, info.as_dict()
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-6
    G.close()


def test_bounded_wait_gives_up_with_timeout_then_recovers():
    """Failure detection of the tensor-core kernel's pipeline (not in the
    paper).  With the pipeline waits limited to 1 ns a wait gives up: the
    kernel stops writing, drains its own copies and products (full limit),
    frees its tensor memory and sets the problem's error word, which
    wc4d_status reports as WC4D_ERR_TIMEOUT (and clears).  With the default
    limit restored the same problem applies A to 1e-11 of the oracle and
    solves to the true residual: the context and the problem stay usable."""
    w, dr = case(512, 40, 256, seed=6)
    prob, obs, rhs = prb.linear_case(w, dr)
    G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=3, precision="ozaki", tol=1e-8, maxit=500))
    v = W.random_vector(prob.n, 9)
    want = prob.A_apply(v)
    codes = []
    try:
        L.wc4d_set_wait_limit_ns(1)
        for _ in range(3):
            G.apply_saddle(to_dev(v))
            codes.append(L.wc4d_status(G.h, raise_on_error=False))
            if codes[-1] == L.WC4D_ERR_TIMEOUT:
                break
    finally:
        L.wc4d_set_wait_limit_ns(0)
    assert L.WC4D_ERR_TIMEOUT in codes, codes
    assert "bounded wait gave up" in L.wc4d_last_error()
    # the word was cleared by the read: the next check is clean
    assert L.wc4d_status(G.h, raise_on_error=False) == L.WC4D_OK
    got = G.apply_saddle(to_dev(v)).cpu().numpy()
    assert L.wc4d_status(G.h, raise_on_error=False) == L.WC4D_OK
    assert rel(got, want) < 1e-11
    x, info = G.solve(to_dev(rhs))
    assert info.status == 0
    r = rhs - prob.A_apply(x.cpu().numpy())
    assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-8
    G.close()


@pytest.mark.parametrize("rhat,kappa", [("rr", 100.0), ("me", 1e4)])
def test_reduced_digit_preconditioner_products(rhat, kappa):
    """prec_digits = d < 7 (not in the paper): the preconditioner's tensor-core
    products keep the leading d BF16 digits of each operand (about 7d - 1 bits,
    d = 1 being BF16 inputs, d = 3 about FP32) with exact FP32 accumulation.
    P_I^{-1} v then differs from the oracle by about kappa(Rhat) 2^(2 - 7d)
    (Rhat reconditioned to kappa_max by Alg. 1 / 2, Sec. 5.2), and the error
    falls by about 2^7 per digit.  The flexible GMRES (preconditioned vectors
    kept) still reaches an FP64 true residual of 1e-8 (below the paper's 1e-6)
    with the oracle's operator, in at most twice the iterations of the 7-digit
    products; its forward error against dense LU is reported.  (Pushed to 1e-10
    the 3-digit solve stagnates near 3e-10 within 1500 iterations.)"""
    w, dr = case(256, 12, 128, seed=8)
    prob, obs, rhs = prb.linear_case(w, dr)
    x_lu = sd.dense_solve(prob, rhs)
    P = sd.Preconditioner(prob, sd.PrecondOptions(kind="PI", k=3, rhat=rhat, kappa_max=kappa))
    v = W.random_vector(prob.n, 10)
    ref = P.apply(v)
    errs = {}
    for d in (2, 3, 4, 7):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=3, rhat=rhat, kappa_max=kappa,
                                                       precision="ozaki", prec_digits=d))
        errs[d] = rel(G.apply_precond("PI", to_dev(v)).cpu().numpy(), ref)
        # A v keeps all 7 digits whatever the preconditioner uses
        assert rel(G.apply_saddle(to_dev(v)).cpu().numpy(), prob.A_apply(v)) < 1e-11
        G.close()
    assert errs[7] < 1e-9
    for d in (2, 3, 4):
        assert errs[d] < 4.0 * kappa * 2.0 ** (2 - 7 * d), errs
    assert errs[2] > errs[3] > errs[4] > errs[7], errs
    its = {}
    for d in (3, 7):
        G = L.Problem.from_workload(w, dr, L.make_opts(precond="PI", k=3, rhat=rhat, kappa_max=kappa,
                                                       precision="ozaki", prec_digits=d, tol=1e-8, maxit=1500))
        x, info = G.solve(to_dev(rhs))
        assert info.status == 0, (d, L.wc4d_last_error())
        r = rhs - prob.A_apply(x.cpu().numpy())
        assert np.linalg.norm(r) / np.linalg.norm(rhs) <= 1e-8
        its[d] = info.iters
        fwd = rel(x.cpu().numpy(), x_lu)
        print(f"prec_digits={d} rhat={rhat} kappa_max={kappa}: {info.iters} iterations, "
              f"forward error vs LU {fwd:.2e}")
        assert fwd < 1e-4   # kappa(A) (~1e5 here) times the 1e-8 residual, with margin
        G.close()
    assert its[3] <= 2 * its[7] + 5, its


def test_reduced_digits_need_ozaki_gmres():
    w, dr = case(64, 3, 32, seed=1)
    for kw in ({"precision": "df32"}, {"precision": "ozaki", "precond": "PD", "krylov": "minres"}):
        with pytest.raises(L.WC4DError) as e:
            L.Problem.from_workload(w, dr, L.make_opts(**{"precond": "PI", "k": 2, "prec_digits": 3, **kw}))
        assert e.value.code == L.WC4D_ERR_ARG and "reduced-digit" in str(e.value)
