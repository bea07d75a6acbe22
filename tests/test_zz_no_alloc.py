"""spamm_leaf_sqnorms_noalloc: the entry point for callers that must not
allocate device memory (services that reserve all device memory up front,
plug-ins inside a framework that owns the device memory).  Its results must
match what the allocating entry points compute for the same leaves, on two
calls in a row sharing the library's fixed scratch array."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL_NORM = 1e-14  # the norm tolerance of the other GPU tests


@pytest.fixture(scope="module")
def S():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_1906_08148_gb300 import spamm
    return spamm


@pytest.mark.parametrize("bs,p", [(64, synth.lattice_3d(16384, alpha=0.9, seed=5)),
                                  (32, synth.model_1d(20000, alpha=0.02, seed=6))])
def test_noalloc_matches_the_allocating_entry_points(S, bs, p):
    import torch
    with S.Context(0) as ctx:
        G = S.spamm_generate(ctx, p, bs)
        bi, bj, pay, sq_ref = S.spamm_to_blocks(ctx, G)
        total_ref = S.spamm_frob_norm(ctx, G) ** 2
        G.close()
    nl = len(bi)
    assert nl > 4096  # several scratch partials
    payload = torch.from_numpy(pay).cuda()
    stream = torch.cuda.current_stream()
    for call in range(2):
        sq = torch.full((nl,), -1.0, dtype=torch.float64, device="cuda")
        total = torch.full((1,), -1.0, dtype=torch.float64, device="cuda")
        st = S.spamm_leaf_sqnorms_noalloc(payload, nl, bs, sq, total, stream)
        assert st == S.OK, st
        torch.cuda.synchronize()
        got = sq.cpu().numpy()
        # the same per-leaf arithmetic and order as the library's norm pass: identical bits
        assert np.array_equal(got, sq_ref), call
        # the total adds the partial sums in another order than the quadtree's parents
        assert abs(float(total.item()) - total_ref) <= REL_NORM * total_ref, call


def test_noalloc_second_call_with_fewer_leaves_and_limits(S):
    import torch
    rng = np.random.default_rng(2)
    pay = rng.standard_normal((9000, 32, 32))
    ref = np.einsum("qij,qij->q", pay, pay)
    payload = torch.from_numpy(pay).cuda()
    sq = torch.empty(9000, dtype=torch.float64, device="cuda")
    total = torch.empty(1, dtype=torch.float64, device="cuda")
    for nl in (9000, 100, 0):  # later calls use fewer scratch entries than earlier ones
        assert S.spamm_leaf_sqnorms_noalloc(payload, nl, 32, sq, total, None) == S.OK
        torch.cuda.synchronize()
        want = float(np.sum(ref[:nl]))
        assert abs(float(total.item()) - want) <= 1e-13 * max(want, 1.0)
        if nl:
            assert np.allclose(sq.cpu().numpy()[:nl], ref[:nl], rtol=1e-13)
    # the library's own limits, reached with raw pointers (the binding checks
    # tensor sizes first; the library refuses these before anything is enqueued)
    p, q, t = payload.data_ptr(), sq.data_ptr(), total.data_ptr()
    assert S.spamm_leaf_sqnorms_noalloc(p, S.NOALLOC_MAX_LEAVES + 1, 32, q, t, None) == S.E_CAPACITY
    assert S.spamm_leaf_sqnorms_noalloc(p, 10, 48, q, t, None) == S.E_INVALID_ARG
    with pytest.raises(ValueError):
        S.spamm_leaf_sqnorms_noalloc(payload, S.NOALLOC_MAX_LEAVES + 1, 32, sq, total, None)


def test_noalloc_refuses_misaligned_or_wrong_buffers_on_the_host(S):
    """Misaligned raw pointers get INVALID_ARG from the library's host-side
    check (nothing is enqueued); wrong tensors are refused by the binding."""
    import torch
    pay = torch.zeros(4 * 32 * 32 + 2, dtype=torch.float64, device="cuda")
    sq = torch.zeros(8, dtype=torch.float64, device="cuda")
    total = torch.zeros(2, dtype=torch.float64, device="cuda")
    base = pay.data_ptr()
    assert base % 16 == 0
    assert S.spamm_leaf_sqnorms_noalloc(base + 8, 4, 32, sq.data_ptr(), total.data_ptr(), None) == S.E_INVALID_ARG
    assert S.spamm_leaf_sqnorms_noalloc(base, 4, 32, sq.data_ptr() + 4, total.data_ptr(), None) == S.E_INVALID_ARG
    assert S.spamm_leaf_sqnorms_noalloc(base, 4, 32, sq.data_ptr(), total.data_ptr() + 4, None) == S.E_INVALID_ARG
    torch.cuda.synchronize()
    assert float(sq.abs().sum().item()) == 0.0  # nothing ran
    with pytest.raises(ValueError):
        S.spamm_leaf_sqnorms_noalloc(pay.float(), 4, 32, sq, total)
    with pytest.raises(ValueError):
        S.spamm_leaf_sqnorms_noalloc(pay.cpu(), 4, 32, sq, total)
    with pytest.raises(ValueError):
        S.spamm_leaf_sqnorms_noalloc(pay[:100], 4, 32, sq, total)
    with pytest.raises(ValueError):
        S.spamm_leaf_sqnorms_noalloc(pay[: 4 * 1024 * 2].view(-1, 2)[:, 0], 4, 32, sq, total)
    assert S.spamm_leaf_sqnorms_noalloc(pay, 4, 32, sq, total) == S.OK
