"""stst_rhs_noalloc, the right-hand side for callers that cannot allocate device memory.

Those callers (code recorded during CUDA stream capture, where cudaMalloc and
cudaFree are forbidden, and programs whose device memory is already held by
their own pool or budget) get the same vector as stst_rhs, computed in a
static scratch array built into the library instead of call-time
allocations. This file is collected last so that a failure here comes after
every other test has run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2311_18461_gb300 as S
from inputs import harmonic_potential, wavepacket_factors, wavepacket_params
from tests._common import rel_err, sample_potential, sample_initial, sample_forcing, to_np

pytestmark = pytest.mark.gpu


def _forcing(t, *xs):
    return np.exp(1j * (2 * t + xs[0])) * (1 + 0.5 * sum(x ** 2 for x in xs))


@pytest.mark.parametrize("n_el,p,with_potential,form", [
    ([6, 7, 5], [2, 2, 3], True, S.STST_FORM_LS),
    ([9, 8], [3, 2], False, S.STST_FORM_LS),
    ([6, 7, 5], [2, 2, 3], True, S.STST_FORM_UW),     # the ultraweak load: T0 only, initial term added
    ([4, 5, 4, 3], [2, 2, 3, 2], True, S.STST_FORM_LS),  # 3D+t: the chain of contractions through W1, W2
])
def test_noalloc_matches_allocating_rhs_on_consecutive_calls(n_el, p, with_potential, form):
    d = len(n_el) - 1
    prob = S.Problem(d, n_el, p, T=0.8, nu=1.2, formulation=form)
    if with_potential:
        V = harmonic_potential(d)
        prob.set_potential(sample_potential(prob, V), len(V))
    u0 = wavepacket_factors(wavepacket_params(np.random.default_rng(3), d))
    f_qp = sample_forcing(prob, _forcing)
    u0_qp = sample_initial(prob, u0)
    ref, c_ref = prob.rhs(f_qp, u0_qp, want_c0=True)
    torch.cuda.synchronize()
    for _ in range(2):  # the shared scratch keeps the previous call's contents
        out = torch.full_like(ref, complex(7.0, -3.0))
        c0 = torch.full_like(c_ref, complex(-1.0, 2.0))
        S.stst_rhs_noalloc(prob.h, f_qp, u0_qp, out, c0)
        torch.cuda.synchronize()
        assert rel_err(to_np(out), to_np(ref)) < 1e-12
        assert rel_err(to_np(c0), to_np(c_ref)) < 1e-12
    # forcing only, then initial datum only
    out = prob.vec()
    S.stst_rhs_noalloc(prob.h, f_qp, None, out, None)
    ref_f = prob.vec()
    S.stst_rhs(prob.h, f_qp, None, ref_f, None)
    torch.cuda.synchronize()
    assert rel_err(to_np(out), to_np(ref_f)) < 1e-12
    prob.close()


def test_noalloc_takes_no_device_memory_and_rejects_oversized_grids():
    prob = S.Problem(1, [6, 7], [2, 3])
    f_qp = sample_forcing(prob, _forcing)
    out = prob.vec()
    S.stst_rhs_noalloc(prob.h, f_qp, None, out, None)   # first call on the device: address lookup
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        S.stst_rhs_noalloc(prob.h, f_qp, None, out, None)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    prob.close()
    # 4 * n_t * Q_1 * Q_2 complex values exceed the 2^20 of the static array
    big = S.Problem(2, [60, 40, 40], [2, 2, 2])
    assert 4 * big.n[0] * (40 * 4) ** 2 > 2 ** 20
    f_big = torch.zeros(60 * 4 * (40 * 4) ** 2, dtype=torch.complex128, device="cuda")
    with pytest.raises(S.StstError) as e:
        S.stst_rhs_noalloc(big.h, f_big, None, big.vec(), None)
    assert e.value.status == -1
    big.close()


def test_noalloc_ultraweak_load_needs_three_slices():
    """The ultraweak load uses three grid-sized slices of the static array (no least-squares time
    derivative, no potential term): a grid that needs 3 but not 4 or 5 slices is accepted, with a
    potential installed, and matches stst_rhs."""
    n_el, p = [30, 25, 25], [2, 2, 2]
    prob = S.Problem(2, n_el, p, formulation=S.STST_FORM_UW)
    sz = prob.n[0] * (25 * 4) ** 2
    assert 3 * sz <= 2 ** 20 < 4 * sz
    V = harmonic_potential(2)
    prob.set_potential(sample_potential(prob, V), len(V))
    f_qp = sample_forcing(prob, _forcing)
    ref = prob.vec()
    S.stst_rhs(prob.h, f_qp, None, ref, None)
    for _ in range(2):
        out = torch.full_like(ref, complex(5.0, 1.0))
        S.stst_rhs_noalloc(prob.h, f_qp, None, out, None)
        torch.cuda.synchronize()
        assert rel_err(to_np(out), to_np(ref)) < 1e-12
    prob.close()
