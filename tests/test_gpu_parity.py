"""Parity of the CUDA library (through its C ABI) with the FP64 CPU oracle.

Tolerances: FP64 path 1e-12 relative (operators) and 1e-10 (PCG iterates,
the same algorithm in the same order); FP32 preconditioner 1e-5 relative on
P-hat^{-1} r; solutions of the mixed path within 1e-8 of the FP64 oracle's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, bump_potential, wavepacket_factors, wavepacket_params, random_complex
from oracle import fd as ofd, pcg as opcg, rhs as orhs, matrices as omat
from tests._common import (rel_err, oracle_disc, sample_potential, sample_initial, sample_forcing, to_dev, to_np)

pytestmark = pytest.mark.gpu

CASES = [
    # (n_el, p, potential)
    ([32, 32], 2, None),
    ([7, 9], [1, 3], None),
    ([9, 11, 7], [2, 3, 2], None),
    ([9, 11, 7], [2, 3, 3], "harmonic"),
    ([5, 6, 5, 7], [2, 2, 3, 2], None),
    ([5, 6, 5, 4], [3, 2, 2, 2], "bump"),
    ([3, 1], [1, 2], None),
    # harmonic potentials in 1D+t and 3D+t: the mat-vec's grouped form for sums of one-direction factors
    ([6, 9], [2, 3], "harmonic"),
    ([5, 6, 5, 4], [2, 2, 3, 2], "harmonic"),
]


def _pot(kind, d):
    if kind is None:
        return None
    return harmonic_potential(d) if kind == "harmonic" else bump_potential(d)


def _problem(n_el, p, kind, prec=S.STST_PREC_FP64, T=1.0, nu=1.0):
    d = len(n_el) - 1
    pl = [p] * (d + 1) if isinstance(p, int) else list(p)
    prob = S.Problem(d, n_el, pl, T=T, nu=nu, prec_mode=prec)
    V = _pot(kind, d)
    if V is not None:
        prob.set_potential(sample_potential(prob, V), len(V))
    disc = oracle_disc(n_el, pl, T=T, nu=nu, potential=V)
    return prob, disc


def _band_to_dense(band, n, p):
    A = np.zeros((n, n))
    for i in range(n):
        for k in range(2 * p + 1):
            j = i - p + k
            if 0 <= j < n:
                A[i, j] = band[i * (2 * p + 1) + k]
    return A


@pytest.mark.parametrize("p,n_el,length,bc", [(2, 5, 1.0, 2), (3, 9, 2.0, 1), (4, 6, 0.7, 0), (1, 4, 1.3, 1),
                                              (8, 3, 1.0, 2)])
def test_assemble_1d(p, n_el, length, bc):
    m = n_el + p
    n = m - bc
    bufs = [torch.zeros(n * (2 * p + 1), dtype=torch.float64, device="cuda") for _ in range(5)]
    assert S.stst_assemble_1d(p, n_el, length, bc, None, *bufs) == n
    torch.cuda.synchronize()
    F = omat.assemble_1d(p, n_el, length)
    sl = {0: slice(0, m), 1: slice(1, m), 2: slice(1, m - 1)}[bc]
    for key, b in zip(["M", "L", "J", "K", "K2"], bufs):
        ref = F[key][sl, sl]
        got = _band_to_dense(to_np(b), n, p)
        assert rel_err(got, ref) < 1e-13, key


def test_quadrature_points():
    prob, disc = _problem([4, 6, 5], [2, 3, 4], None, T=1.7)
    for l in range(prob.d + 1):
        np.testing.assert_allclose(to_np(prob.quad_points(l)), disc.quad(l)[0], rtol=0, atol=1e-14)


@pytest.mark.parametrize("n_el,p,kind", CASES)
def test_apply_sys(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind, T=1.3, nu=0.8)
    x = random_complex(prob.n_dof, 11)
    y = to_np(prob.apply_sys(to_dev(x)))
    ref = disc.apply(x)
    assert rel_err(y, ref) < 1e-12


@pytest.mark.parametrize("n_el,p,kind", CASES)
def test_apply_prec_fp64(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind, T=0.9, nu=1.1)
    assert prob.build_fd() == 0
    r = random_complex(prob.n_dof, 12)
    s = to_np(prob.apply_prec(to_dev(r)))
    ref = ofd.FastDiagonalization(disc).apply(r)
    assert rel_err(s, ref) < 1e-11


@pytest.mark.parametrize("n_el,p", [([9, 11, 7], [2, 3, 2]), ([5, 6, 5, 7], [2, 2, 3, 2]), ([32, 32], 2)])
def test_apply_prec_fp32(n_el, p):
    prob, disc = _problem(n_el, p, None, prec=S.STST_PREC_FP32)
    prob.build_fd()
    r = random_complex(prob.n_dof, 13)
    s = to_np(prob.apply_prec(to_dev(r)))
    ref = ofd.FastDiagonalization(disc).apply(r)
    # FP32 (u = 6e-8): the mode products accumulate n_l <= 128 terms (n u ~ 1e-5 at worst) and the
    # banded solves lose kappa(H_i) ~ 1e2 (u kappa ~ 1e-5): the FD apply is good to a few 1e-5
    assert rel_err(s, ref) < 5e-5


@pytest.mark.parametrize("n_el,p", [([9, 11, 7], [2, 3, 2]), ([5, 6, 5, 7], [2, 2, 3, 2]), ([32, 32], 2),
                                   ([6, 126], [2, 4]), ([64, 64, 64], [3, 3, 3])])
def test_apply_prec_bf16_tensor_cores(n_el, p):
    """Mode products on tcgen05 tensor cores: BF16 operands split into high and low parts, FP32 accumulation."""
    prob, disc = _problem(n_el, p, None, prec=S.STST_PREC_BF16)
    prob.build_fd()
    r = random_complex(prob.n_dof, 14)
    s = to_np(prob.apply_prec(to_dev(r)))
    ref = ofd.FastDiagonalization(disc).apply(r)
    # with x = x_hi + x_lo and U = U_hi + U_lo in BF16 the three products keep ~16 significant bits
    # (dropped x_lo U_lo and the lo rounding are ~2^-17 relative), the FP32 time solves lose
    # kappa(H_i) ~ 1e2 times FP32 rounding: the FD apply is good to about 1e-4 relative
    assert rel_err(s, ref) < 1e-4


@pytest.mark.parametrize("n_el,p,kind", [([9, 11, 7], [2, 3, 2], "harmonic"), ([5, 6, 5, 7], [2, 2, 3, 2], None)])
def test_pcg_bf16_preconditioner_solution(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind, prec=S.STST_PREC_BF16)
    prob.build_fd()
    b = random_complex(prob.n_dof, 24)
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=300)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-13, maxit=300)
    assert st == 0
    assert rel_err(to_np(x), xo) < 1e-8


@pytest.mark.parametrize("n_el,p,kind", [([8, 9], [2, 3], None), ([6, 7, 5], [2, 2, 3], "harmonic"),
                                         ([4, 5, 4, 3], 2, "bump")])
def test_rhs_lifting_and_forcing(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind, T=0.8, nu=1.2)
    d = prob.d
    wp = wavepacket_factors(wavepacket_params(np.random.default_rng(3), d))
    f = lambda t, *xs: np.exp(1j * (2 * t + xs[0])) * (1 + 0.5 * sum(x ** 2 for x in xs))
    b_gpu, c_gpu = prob.rhs(sample_forcing(prob, f), sample_initial(prob, wp), want_c0=True)
    from inputs import product_fn
    b_ref, c_ref = orhs.rhs_initial(disc, f, product_fn(wp))
    assert rel_err(to_np(c_gpu), c_ref.ravel()) < 1e-12
    assert rel_err(to_np(b_gpu), b_ref) < 1e-12


@pytest.mark.parametrize("n_el,p,kind", CASES[:6])
def test_pcg_fp64_matches_oracle_iterates(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind)
    prob.build_fd()
    b = random_complex(prob.n_dof, 21)
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-10, maxit=200)
    F = ofd.FastDiagonalization(disc)
    xo, ito, rro, _ = opcg.pcg(disc.apply, F.apply, b, tol=1e-10, maxit=200)
    assert st == 0 and rr <= 1e-10
    assert abs(it - ito) <= 1
    assert rel_err(to_np(x), xo) < 1e-9
    # residual of the GPU solution measured by the oracle
    res = np.linalg.norm(b - disc.apply(to_np(x))) / np.linalg.norm(b)
    assert res < 1e-9


@pytest.mark.parametrize("where", ["last", "first", "middle"])
def test_pcg_nonzero_initial_guess_follows_the_oracle(where):
    """From x0 = 0 the residual is f without a mat-vec (a device check of x0); any nonzero entry of x0,
    wherever it sits in the vector, must send the solve through r = f - A x0: the iterates then follow
    the oracle's PCG from the same x0 (FP64 path)."""
    prob, disc = _problem([9, 11, 7], [2, 3, 2], "harmonic")
    prob.build_fd()
    b = random_complex(prob.n_dof, 27)
    x0 = np.zeros(prob.n_dof, dtype=complex)
    k = {"last": prob.n_dof - 1, "first": 0, "middle": prob.n_dof // 2 + 3}[where]
    x0[k] = 0.7 - 0.2j
    xd = to_dev(x0)
    x, st, it, rr = prob.pcg(to_dev(b), xd, tol=1e-10, maxit=200)
    F = ofd.FastDiagonalization(disc)
    xo, ito, rro, _ = opcg.pcg(disc.apply, F.apply, b, x0=x0, tol=1e-10, maxit=200)
    assert st == 0 and abs(it - ito) <= 1
    assert rel_err(to_np(x), xo) < 1e-9
    # the same solve from zero takes the zero-guess path and still matches the oracle from zero
    x, st, it0, rr = prob.pcg(to_dev(b), None, tol=1e-10, maxit=200)
    xo0, ito0, _, _ = opcg.pcg(disc.apply, F.apply, b, tol=1e-10, maxit=200)
    assert st == 0 and abs(it0 - ito0) <= 1 and rel_err(to_np(x), xo0) < 1e-9


def test_profile_counts_kernels_and_graph_body_holds_two_iterations():
    """The tracing hook counts kernel launches (a record may time a short run of them), and the PCG
    graph's WHILE body holds two iterations of the plain loop: two more plain iterations launch
    exactly one body's kernel nodes."""
    prob, disc = _problem([9, 11, 7], [2, 3, 2], "harmonic", prec=S.STST_PREC_FP32)
    prob.build_fd()
    b = to_dev(random_complex(prob.n_dof, 31))
    x = prob.vec()
    with pytest.raises(S.StstError):
        S.stst_pcg_graph_info(prob.h)  # the graph is built by the first unprofiled solve
    counts = []
    for maxit in (1, 3):
        x.zero_()
        S.stst_profile(prob.h, 1)
        st, it, rr = S.stst_pcg_solve(prob.h, b, x, 1e-14, maxit)
        prof = S.stst_profile_read(prob.h)
        S.stst_profile(prob.h, 0)
        assert st == S.STST_NOT_CONVERGED and it == maxit
        assert prof["pcg_update_xr"][0] == maxit and prof["pcg_init"][0] == 5
        counts.append(sum(c for c, _ in prof.values()))
    x.zero_()
    st, it, rr = S.stst_pcg_solve(prob.h, b, x, 1e-10, 200)
    assert st == 0
    kpb, ipb = S.stst_pcg_graph_info(prob.h)
    assert ipb == 2 and kpb == counts[1] - counts[0]
    prob.close()


@pytest.mark.parametrize("n_el,p,kind", [([9, 11, 7], [2, 3, 2], "harmonic"), ([5, 6, 5, 7], [2, 2, 3, 2], None)])
def test_pcg_fp32_preconditioner_solution(n_el, p, kind):
    prob, disc = _problem(n_el, p, kind, prec=S.STST_PREC_FP32)
    prob.build_fd()
    b = random_complex(prob.n_dof, 22)
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=200)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-12, maxit=200)
    assert st == 0
    assert rel_err(to_np(x), xo) < 1e-8


@pytest.mark.parametrize("n_el,p,kind", [([9, 11, 7], [2, 3, 2], "harmonic"), ([5, 6, 5, 7], [2, 2, 3, 2], None),
                                         ([32, 32], 2, None)])
def test_iterative_refinement_solution(n_el, p, kind):
    """FP64 residual/update around FP32 inner PCG: final solution within 1e-8 of the FP64 oracle's."""
    prob, disc = _problem(n_el, p, kind, prec=S.STST_PREC_FP32)
    prob.build_fd()
    b = random_complex(prob.n_dof, 23)
    x, st, it, outer, rr = prob.ir(to_dev(b), tol=1e-10, maxit=80, inner_tol=1e-4, inner_maxit=100)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-13, maxit=300)
    assert st == 0 and rr <= 1e-10
    assert rel_err(to_np(x), xo) < 1e-8
    res = np.linalg.norm(b - disc.apply(to_np(x))) / np.linalg.norm(b)
    assert res < 1e-9


def test_iterative_refinement_degenerate_starts():
    """IR started at the solution stops after its first FP64 residual, with no inner solve and x untouched;
    maxit = 0 only measures the residual of the start (x0 = 0: relative residual 1)."""
    prob, disc = _problem([9, 11, 7], [2, 3, 2], "harmonic", prec=S.STST_PREC_FP32)
    prob.build_fd()
    b = random_complex(prob.n_dof, 24)
    xo, _, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-13, maxit=300)
    x, st, it, outer, rr = prob.ir(to_dev(b), to_dev(xo), tol=1e-10, maxit=10)
    assert st == 0 and outer == 0 and it == 0 and rr <= 1e-10
    assert np.array_equal(to_np(x), xo)
    x, st, it, outer, rr = prob.ir(to_dev(b), None, tol=1e-10, maxit=0)
    assert st == S.STST_NOT_CONVERGED and outer == 0 and it == 0
    assert abs(rr - 1.0) < 1e-12 and not np.any(to_np(x))


def test_c1_workload_end_to_end():
    """1D+t, p=2, 32x32, u = exp(i pi^2 t) sin(pi x): rhs by lifting, PCG to 1e-10, against the oracle."""
    from inputs import CONFIGS, initial_factors, product_fn
    cfg = CONFIGS["c1"]
    prob, disc = _problem(cfg["n_el"], cfg["p"], None)
    u0 = initial_factors(cfg)
    b, c0 = prob.rhs(None, sample_initial(prob, u0), want_c0=True)
    b_ref, c_ref = orhs.rhs_initial(disc, None, product_fn(u0))
    # the lifted rhs is a difference of terms about 1e4 times larger than the result (nu^2 J_l c with
    # J ~ h^-3): FP64 rounding in a different summation order shows at ~1e-12 relative to max|rhs|
    assert rel_err(to_np(b), b_ref) < 1e-11
    prob.build_fd()
    x, st, it, rr = prob.pcg(b, tol=cfg["tol"], maxit=200)
    xo, ito, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b_ref, tol=cfg["tol"])
    assert st == 0 and abs(it - ito) <= 1
    assert rel_err(to_np(x), xo) < 1e-9


# ---------------------------------------------------------------------------------------- edge cases
def test_degenerate_sizes():
    # one spatial unknown, one time unknown
    prob, disc = _problem([1, 1], [1, 2], None)
    assert prob.n_dof == 1
    prob.build_fd()
    x = random_complex(1, 1)
    assert rel_err(to_np(prob.apply_sys(to_dev(x))), disc.apply(x)) < 1e-13
    xs, st, it, rr = prob.pcg(to_dev(x), tol=1e-12)
    assert st == 0 and it <= 1


def test_max_space_size_and_degree():
    prob, disc = _problem([3, 126], [2, 4], None)  # n_1 = 128
    prob.build_fd()
    r = random_complex(prob.n_dof, 5)
    assert rel_err(to_np(prob.apply_prec(to_dev(r))), ofd.FastDiagonalization(disc).apply(r)) < 1e-10
    prob8, disc8 = _problem([3, 4], [1, 8], None)
    prob8.build_fd()
    r = random_complex(prob8.n_dof, 6)
    assert rel_err(to_np(prob8.apply_prec(to_dev(r))), ofd.FastDiagonalization(disc8).apply(r)) < 1e-10


def test_status_codes():
    with pytest.raises(S.StstError):
        S.Problem(2, [4, 4, 4], [2, 1, 2])  # p_s = 1 violates C^1 in space
    with pytest.raises(S.StstError):
        S.Problem(1, [4, 200], [2, 2])       # n_s > 128
    with pytest.raises(S.StstError):
        S.Problem(0, [4], [2])
    prob, _ = _problem([4, 5], 2, None)
    r = prob.vec()
    with pytest.raises(S.StstError) as e:
        prob.apply_prec(r)                   # before build_fd
    assert e.value.status == -5
    with pytest.raises(S.StstError):
        S._lib._chk(S.lib().stst_apply_sys(None, r.data_ptr(), r.data_ptr()), "x")
    prob.build_fd()
    b = to_dev(random_complex(prob.n_dof, 9))
    x, st, it, rr = prob.pcg(b, tol=0.0, maxit=3)
    assert st == 1 and it == 3
    x, st, it, rr = prob.pcg(b, tol=1e-8, maxit=0)
    assert st == 1 and it == 0 and np.abs(to_np(x)).max() == 0
    bn = b.clone()
    bn[0] = complex(float("nan"), 0)
    x, st, it, rr = prob.pcg(bn, tol=1e-8, maxit=10)
    assert st in (1, 2)
    # zero right-hand side: converged immediately with x = 0
    x, st, it, rr = prob.pcg(prob.vec(), tol=1e-8, maxit=10)
    assert st == 0 and it == 0


def test_rejected_potential_keeps_the_previous_operator():
    """A potential with a non-finite sample is rejected (STST_ERR_ARG) before anything of the handle
    changes: the mat-vec, the captured PCG graph and the iterative-refinement graph keep applying the
    potential installed before, and a later valid potential replaces it in all of them."""
    prob, disc = _problem([6, 7, 5], [2, 3, 2], "harmonic", prec=S.STST_PREC_FP32)
    prob.build_fd()
    b = random_complex(prob.n_dof, 61)
    x1, st, _, _ = prob.pcg(to_dev(b), tol=1e-10, maxit=200)      # builds the PCG graph
    y1, st1, _, _, _ = prob.ir(to_dev(b), tol=1e-10, maxit=40)     # builds the IR graph
    assert st == 0 and st1 == 0
    bad = sample_potential(prob, harmonic_potential(2))
    bad[3] = float("nan")
    with pytest.raises(S.StstError) as e:
        prob.set_potential(bad, 2)
    assert e.value.status == S.STST_ERR_ARG
    v = random_complex(prob.n_dof, 62)
    assert rel_err(to_np(prob.apply_sys(to_dev(v))), disc.apply(v)) < 1e-12
    x2, st, _, _ = prob.pcg(to_dev(b), tol=1e-10, maxit=200)
    assert st == 0 and rel_err(to_np(x2), to_np(x1)) < 1e-12
    # a different valid potential reaches the mat-vec and both solver graphs
    V = bump_potential(2)
    prob.set_potential(sample_potential(prob, V), len(V))
    disc_b = oracle_disc([6, 7, 5], [2, 3, 2], potential=V)
    assert rel_err(to_np(prob.apply_sys(to_dev(v))), disc_b.apply(v)) < 1e-12
    xo, _, _, _ = opcg.pcg(disc_b.apply, ofd.FastDiagonalization(disc_b).apply, b, tol=1e-13, maxit=300)
    x3, st, _, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=300)
    assert st == 0 and rel_err(to_np(x3), xo) < 1e-8
    y3, st, _, _, _ = prob.ir(to_dev(b), tol=1e-10, maxit=80, inner_maxit=100)
    assert st == 0 and rel_err(to_np(y3), xo) < 1e-8
    prob.close()


@pytest.mark.parametrize("p", [2, 3, 4])
def test_apply_prec_size_sweep(p):
    """Every spatial size from 1 to 100 unknowns: the eigen setup must handle the nearly degenerate
    pairs of boundary outlier eigenvalues of the B-spline pencils (all three precisions)."""
    bad = []
    for n_el in list(range(1, 40)) + list(range(40, 100, 7)):
        if n_el + p - 2 < 1:
            continue
        disc = oracle_disc([3, n_el], [2, p])
        ref_fd = ofd.FastDiagonalization(disc)
        r = random_complex(disc.N_dof, 15)
        ref = ref_fd.apply(r)
        for prec, tol in [(S.STST_PREC_FP64, 1e-10), (S.STST_PREC_FP32, 5e-5), (S.STST_PREC_BF16, 1e-4)]:
            prob = S.Problem(1, [3, n_el], [2, p], prec_mode=prec)
            assert prob.build_fd() == 0
            err = rel_err(to_np(prob.apply_prec(to_dev(r))), ref)
            if err > tol:
                bad.append((n_el, prec, err))
            prob.close()
    assert not bad, bad


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [0, 1])
def test_mode_product_tiles_agree_bitwise(prec):
    """Every mode-product tile sums each output in the same order: apply_prec is bitwise identical."""
    import torch
    import paper_2311_18461_gb300 as P
    outs = {}
    P.stst_set_time_solver(1)  # the same time solve for every tile
    P.stst_set_fused_transforms(1)  # separate mode products, so that every tile runs
    P.stst_set_pencil(1)
    P.stst_set_tensor_products(1)  # SIMT tiles only
    try:
        for mode in (0, 12, 14, 22, 24, 32, 34, 42, 44, 132, 1):
            P.stst_set_autotune(mode)
            prob = P.Problem(2, [5, 40, 70], 3, prec_mode=prec)  # n_l = 41 and 71
            prob.build_fd()
            r = torch.tensor(np.random.default_rng(3).standard_normal(2 * prob.n_dof), device="cuda").view(
                torch.complex128)
            outs[mode] = (prob.apply_prec(r).cpu().numpy(), [P.stst_tile_info(prob.h, l) for l in (1, 2)])
            prob.close()
    finally:
        P.stst_set_autotune(1)
        P.stst_set_time_solver(0)
        P.stst_set_fused_transforms(0)
        P.stst_set_pencil(0)
        P.stst_set_tensor_products(0)
    ref = outs[0][0]
    for mode, (o, tiles) in outs.items():
        assert np.array_equal(o, ref), (mode, tiles)
    assert outs[12][1][0][:2] == (16, 32) and outs[44][1][1][:2] == (32, 128)
    if prec == S.STST_PREC_FP32:  # the wide 32-row x 256-column tile (FP32 only)
        assert outs[132][1][0][:2] == (256, 32) and outs[132][1][1][:2] == (256, 32)


@pytest.mark.parametrize("n_el,p", [([5, 40, 70], 3), ([9, 16, 78], [2, 3, 3]), ([3, 1, 5], 2), ([70, 30, 31], 2),
                                    ([5, 12, 9, 7], [2, 3, 2, 2]), ([4, 30, 6, 40], [3, 2, 3, 2])])
def test_fused_2d_transforms_bitwise(n_el, p):
    """The fused transform kernel (the mode products of directions 1 and 2 of Algorithm 1 steps 2 and 4
    in one kernel per (t, x_3) slab; direction 3 separate when d = 3) gives bitwise the same
    preconditioner output as the separate mode-product kernels; PCG with either takes the same
    iterations (only the order of the dot-product partial sums differs). Mode 0 lets the tuner choose,
    which may give the backward transform another split than the forward one."""
    out = {}
    S.stst_set_pencil(1)  # the separate last-direction kernels, so that the fused transforms run for d = 2
    S.stst_set_tensor_products(1)  # the SIMT mode products, which sum in the fused kernel's order
    try:
        for mode in (1, 0, 2, 11, 12, 13, 14):
            S.stst_set_fused_transforms(mode)
            prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=S.STST_PREC_FP32)
            prob.build_fd()
            fused = S.stst_fused_transforms_info(prob.h)
            split = S.stst_fused_transforms_split(prob.h)
            z = to_np(prob.apply_prec(to_dev(random_complex(prob.n_dof, 31))))
            x, st, it, rr = prob.pcg(to_dev(random_complex(prob.n_dof, 32)), tol=1e-10, maxit=300)
            out[mode] = (z, fused, st, it, to_np(x), split)
            prob.close()
    finally:
        S.stst_set_fused_transforms(0)
        S.stst_set_pencil(0)
        S.stst_set_tensor_products(0)
    assert out[1][1] == 0 and out[2][1] >= 1 and out[11][1] == 1
    assert all(out[10 + k][1] in (k, out[2][1]) for k in (2, 3, 4))  # the default where k leaves a part empty
    assert out[1][5] == (0, 0)
    for mode in (2, 11, 12, 13, 14):
        assert out[mode][5] == (out[mode][1], out[mode][1]), (mode, out[mode][5])
    assert out[0][5][0] == out[0][1] and (out[0][5] == (0, 0) or 1 <= out[0][5][1] <= 4), out[0][5]
    for mode in (0, 2, 11, 12, 13, 14):
        assert np.array_equal(out[1][0], out[mode][0]), (mode, out[mode][1])
        assert out[1][2] == 0 and out[mode][2] == 0 and abs(out[1][3] - out[mode][3]) <= 1
        assert rel_err(out[mode][4], out[1][4]) < 1e-8


def test_fused_2d_transforms_only_where_they_apply():
    """Not used with the FP64 or BF16 preconditioners, for d = 1, or when n_1 or n_2 exceeds 80."""
    try:
        S.stst_set_fused_transforms(2)
        for n_el, p, prec in [([4, 6, 7], 2, S.STST_PREC_FP64), ([4, 6, 7], 2, S.STST_PREC_BF16),
                              ([4, 6], 2, S.STST_PREC_FP32), ([3, 4, 90, 6], 2, S.STST_PREC_FP32),
                              ([4, 90, 6], 2, S.STST_PREC_FP32)]:
            prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=prec)
            prob.build_fd()
            assert S.stst_fused_transforms_info(prob.h) == 0, (n_el, prec)
            prob.close()
    finally:
        S.stst_set_fused_transforms(0)
    for bad in (3, 10, 15, -1):
        with pytest.raises(S.StstError):
            S.stst_set_fused_transforms(bad)


@pytest.mark.gpu
@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 1e-4)])
@pytest.mark.parametrize("nt_el,pt", [(3, 1), (8, 2), (33, 3), (64, 3), (40, 4), (97, 2)])
def test_segmented_time_solve_matches_sequential(prec, tol, nt_el, pt):
    """Parallel-in-time (segmented) and sequential time solves agree up to rounding (the segmented form
    reorders the recurrence: zero-start runs plus transfer matrices applied to the carried states)."""
    import torch
    import paper_2311_18461_gb300 as P
    out = {}
    P.stst_set_pencil(1)  # the time-solve kernels (the pencil kernel has its own solves)
    try:
        for mode in (1, 2):
            P.stst_set_time_solver(mode)
            prob = P.Problem(2, [nt_el, 9, 14], [pt, 3, 2], prec_mode=prec)
            prob.build_fd()
            info = P.stst_time_solver_info(prob.h, prec)
            r = torch.tensor(np.random.default_rng(nt_el).standard_normal(2 * prob.n_dof),
                             device="cuda").view(torch.complex128)
            out[mode] = (prob.apply_prec(r).cpu().numpy(), info)
            prob.close()
    finally:
        P.stst_set_time_solver(0)
        P.stst_set_pencil(0)
    assert out[1][1][2] == 0
    if out[2][1][0] >= 2:
        assert out[2][1][2] == 1
    assert rel_err(out[2][0], out[1][0]) < tol, (out[2][1], rel_err(out[2][0], out[1][0]))
