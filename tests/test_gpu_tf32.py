"""Mode products of Algorithm 1 (steps 2 and 4) on the tensor cores: TMA-fed tcgen05 TF32 products, three
per tile (high x high, high x low, low x high), in the FP32 preconditioner.

Each shape is checked against the oracle's FD application and against the same handle type with the SIMT
products. Each term of a product is split into TF32 parts whose three products are good to about 2^-21
relative (near the 2^-24 of the SIMT FMAs), so the two applications agree far below the FP32
preconditioner's own error against the oracle: 1e-5 (measured: about 1e-6). Against the oracle the bound
is the FP32 one of test_apply_prec_fp32 (5e-5), or, where the FP32 preconditioner itself is less accurate
(d = 1 with 66 time and 70 space unknowns: 1.65e-4 with either product), 1.5 times the SIMT path's error.
Shapes: inner extents that are ragged multiples of the 64-column tile, a direction with one unknown, a
direction too large for the kernel's shared memory (it must fall back), odd inner extents (fall back),
and the 3D+t workloads at full size.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, random_complex
from oracle import fd as ofd, pcg as opcg
from tests._common import rel_err, oracle_disc, sample_potential, to_dev, to_np

pytestmark = pytest.mark.gpu


def _inner_extents(n_el, p):
    pl = [p] * len(n_el) if isinstance(p, int) else list(p)
    n = [n_el[0] + pl[0] - 1] + [n_el[l] + pl[l] - 2 for l in range(1, len(n_el))]
    inner, acc = [], n[0]
    for l in range(1, len(n)):
        inner.append(acc)
        acc *= n[l]
    return n, inner


def _expected_dirs(n_el, p):
    """Directions the kernel serves: even inner extent, n_l <= 96, and at least two TMA stages (n_l x 512
    bytes each, 1 KB aligned) with one pair of A planes (128 x K) and the U' planes (N x K) within the
    227 KB of shared memory, less 2 KB for the static part (K = n_l padded to 8, N to 16)."""
    n, inner = _inner_extents(n_el, p)
    mask = 0
    for l in range(1, len(n)):
        nl = n[l]
        npad, kpad = (nl + 15) // 16 * 16, (nl + 7) // 8 * 8
        smem = 2 * ((nl * 512 + 1023) // 1024 * 1024) + 2 * 128 * kpad * 4 + 2 * npad * kpad * 4
        if inner[l - 1] % 2 == 0 and nl <= 96 and smem <= 227 * 1024 - 2048:
            mask |= 1 << l
    return mask


def _build(n_el, p, mode, V=None):
    """A handle with the FP32 preconditioner whose steps 2 and 4 run as separate mode products (the fused 2D
    transforms and the pencil kernel off), with the tensor-core products in the given mode."""
    S.stst_set_tensor_products(mode)
    S.stst_set_fused_transforms(1)
    S.stst_set_pencil(1)
    try:
        prob = S.Problem(len(n_el) - 1, n_el, p, prec_mode=S.STST_PREC_FP32)
        if V is not None:
            prob.set_potential(sample_potential(prob, V), len(V))
        assert prob.build_fd() == 0
    finally:
        S.stst_set_tensor_products(0)
        S.stst_set_fused_transforms(0)
        S.stst_set_pencil(0)
    return prob


SHAPES = [
    ([9, 10, 12], 2),               # n_t = 10: modes 1 (inner 10) and 2 (inner 100 = 64 + 36)
    ([11, 8, 6, 10], [3, 2, 3, 2]),  # n_t = 13: mode 1 odd (SIMT), modes 2 (104) and 3 (728 = 11 x 64 + 24)
    ([65, 70], 2),                  # d = 1, n_1 = 70 (K padded to 72, N to 80), inner 66 = 64 + 2
    ([9, 1, 12], 2),                # a direction with one unknown (K padded from 1 to 8, N to 16)
    ([9, 120], 2),                  # n_1 = 120: the stages exceed shared memory, SIMT products
]


@pytest.mark.parametrize("n_el,p", SHAPES)
def test_tensor_core_products_match_oracle_and_simt(n_el, p):
    prob = _build(n_el, p, 2)
    mask = S.stst_tensor_products_info(prob.h)
    assert mask == _expected_dirs(n_el, p), (mask, _expected_dirs(n_el, p))
    simt = _build(n_el, p, 1)
    assert S.stst_tensor_products_info(simt.h) == 0
    disc = oracle_disc(n_el, p)
    r = random_complex(prob.n_dof, 41)
    s = to_np(prob.apply_prec(to_dev(r)))
    s_simt = to_np(simt.apply_prec(to_dev(r)))
    ref = ofd.FastDiagonalization(disc).apply(r)
    assert rel_err(s, ref) < max(5e-5, 1.5 * rel_err(s_simt, ref))
    assert rel_err(s, s_simt) < 1e-5
    if mask == 0:
        assert np.array_equal(s, s_simt)
    prob.close()
    simt.close()


@pytest.mark.parametrize("n_el,p", [([9, 10, 12], 2), ([11, 8, 6, 10], [3, 2, 3, 2])])
def test_pcg_with_tensor_core_products_reaches_the_oracle_solution(n_el, p):
    """The flexible CG around the FP32 preconditioner (its last product, of direction 1, also forms the
    preconditioned residual's inner products in its epilogue when direction 1 runs on the tensor cores)."""
    V = harmonic_potential(len(n_el) - 1)
    prob = _build(n_el, p, 2, V)
    assert S.stst_tensor_products_info(prob.h) != 0
    disc = oracle_disc(n_el, p, potential=V)
    b = random_complex(prob.n_dof, 42)
    x, st, it, rr = prob.pcg(to_dev(b), tol=1e-12, maxit=200)
    xo, ito, _, _ = opcg.pcg(disc.apply, ofd.FastDiagonalization(disc).apply, b, tol=1e-12, maxit=200)
    assert st == 0
    assert abs(it - ito) <= 2
    assert rel_err(to_np(x), xo) < 1e-8
    prob.close()


def test_autotuned_choice_gives_the_same_application():
    """Mode 0 (the tuner decides per direction) agrees with both forced choices."""
    n_el, p = [11, 8, 6, 10], [3, 2, 3, 2]
    n, _ = _inner_extents(n_el, p)
    r = to_dev(random_complex(int(np.prod(n)), 43))
    outs = {}
    for mode in (0, 1, 2):
        prob = _build(n_el, p, mode)
        outs[mode] = to_np(prob.apply_prec(r))
        prob.close()
    assert rel_err(outs[0], outs[1]) < 1e-5
    assert rel_err(outs[0], outs[2]) < 1e-5


def test_mode_argument_is_checked():
    with pytest.raises(S.StstError):
        S.stst_set_tensor_products(3)
    with pytest.raises(S.StstError):
        S.stst_set_tensor_products(-1)
    S.stst_set_tensor_products(0)


@pytest.mark.parametrize("cfg", ["c3p2", "c3p4"])
def test_full_size_3d_workloads(cfg):
    """The 3D+t workloads at the bench's sizes (32^3 x 64 elements; modes 2 and 3 have even inner extents):
    tensor-core products against the SIMT ones on one random vector."""
    from inputs import CONFIGS
    c = CONFIGS[cfg]
    n_el, p = c["n_el"], c["p"]
    prob = _build(n_el, p, 2)
    assert S.stst_tensor_products_info(prob.h) == _expected_dirs(n_el, p) == 0b1100
    simt = _build(n_el, p, 1)
    gen = torch.Generator(device="cuda").manual_seed(44)
    r = torch.randn(2 * prob.n_dof, dtype=torch.float64, device="cuda", generator=gen).view(torch.complex128)
    s = prob.apply_prec(r)
    s_simt = simt.apply_prec(r)
    err = float((s - s_simt).abs().max() / s_simt.abs().max())
    assert err < 1e-5, err
    prob.close()
    simt.close()
