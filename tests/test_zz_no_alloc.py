"""Allocation-free factorization entry point (stc_factorize_noalloc).

Some callers cannot allocate device memory when they factorize (a service whose own
allocator owns the whole GPU, a real-time loop that must not risk the synchronisation a
cudaMalloc can bring, a plug-in host that only passes buffers in and out).  For them
libstc.so keeps the replay kernel's scratch in a fixed device array; this file checks,
through the C ABI, that two calls in a row give the same factors, log-determinants and
status as the workspace-taking stc_factorize, and that an oversized batch is refused.

It is named to be collected last, and it passes alone in a fresh process as well.
"""
import numpy as np
import pytest

from paper_2609_29765_gb300 import _lib as L
from paper_2609_29765_gb300 import inputs as I
from paper_2609_29765_gb300.api import Plan

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _values(Ap, Ai, seeds):
    return torch.as_tensor(np.stack([I.laplace2d_bordered(seed=s)[2] for s in seeds]), device="cuda")


def test_noalloc_matches_workspace_factorize_twice():
    Ap, Ai, Ax, coords = I.laplace2d_bordered()
    n = len(Ap) - 1
    P = Plan(n, Ap, Ai, coords=coords, nb=64, route="semisparse")
    P.upload()
    batch = 3
    for seeds in ([0, 1, 2], [5, 6, 7]):   # two calls in a row, different values
        v = _values(Ap, Ai, seeds)
        ref = P.factorize(v, check_status=True)
        ref_ld = ref.logdet()
        fac = torch.full((P.factor_bytes(batch) // 8,), float("nan"), dtype=torch.float64, device="cuda")
        info = torch.full((batch,), -7, dtype=torch.int32, device="cuda")
        status = torch.full((1,), -99, dtype=torch.int32, device="cuda")
        rc = L.stc_factorize_noalloc(P.h, v, batch, fac, info, status)
        assert rc == L.STC_OK
        torch.cuda.synchronize()
        assert int(status.item()) == L.STC_OK
        assert torch.equal(info, torch.zeros_like(info))
        ld = torch.empty(batch, dtype=torch.float64, device="cuda")
        assert L.stc_logdet(P.h, fac, batch, ld) == L.STC_OK
        rel = ((ld - ref_ld).abs() / ref_ld.abs()).max().item()
        assert rel <= 1e-10
        Lx = torch.empty(batch, P.nnzL, dtype=torch.float64, device="cuda")
        assert L.stc_factor_to_csc(P.h, fac, batch, Lx) == L.STC_OK
        Lr = ref.to_csc()
        err = ((Lx - Lr).abs().max() / Lr.abs().max()).item()
        assert err <= 1e-12


def test_noalloc_rejects_oversized_batch_and_unuploaded_plan():
    n = 100_000
    Ap, Ai, Ax = I.tridiag(n, 0)
    P = Plan(n, Ap, Ai, nb=8, ordering="natural", route="semisparse")
    ntiles = P.info["ntiles"]
    too_big = (L.STC_NOALLOC_SCRATCH_BYTES - 64) // (4 * ntiles) + 1
    v = torch.zeros(1, P.nnzA, dtype=torch.float64, device="cuda")
    fac = torch.zeros(P.factor_bytes(1) // 8, dtype=torch.float64, device="cuda")
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    # not uploaded yet: refused rather than allocating
    assert L.stc_factorize_noalloc(P.h, v, 1, fac, info) == L.STC_ERR_INVALID_ARG
    P.upload()
    # the size check comes before any launch, so the (small) buffers are never touched
    assert L.stc_factorize_noalloc(P.h, v, too_big, fac, info) == L.STC_ERR_UNSUPPORTED
    vt = torch.as_tensor(Ax, device="cuda")[None].contiguous()
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert L.stc_factorize_noalloc(P.h, vt, 1, fac, info, st) == L.STC_OK
    torch.cuda.synchronize()
    assert int(st.item()) == L.STC_OK and int(info.item()) == 0
    ld = torch.empty(1, dtype=torch.float64, device="cuda")
    assert L.stc_logdet(P.h, fac, 1, ld) == L.STC_OK
    ref = P.factorize(vt).logdet()
    assert abs(ld.item() - ref.item()) <= 1e-10 * abs(ref.item())
