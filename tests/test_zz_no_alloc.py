"""The allocation-free entry point (stiles_factor_selinv_noalloc) gives the
same L, Sigma and logdet as stiles_factor_selinv with a caller-allocated
scratch and as the CPU oracle, on two calls in a row (its fixed scratch array
keeps the previous call's contents), and refuses shapes whose scratch does
not fit the array.

Callers that cannot allocate device memory at call time (a service whose
device memory is reserved once at start-up, code that must not call
cudaMalloc where it runs) use it. This file is collected last on purpose."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err


@pytest.mark.gpu
def test_noalloc_matches_allocating_entry_point_twice():
    S = need_gpu()
    import torch
    M = W.random_arrowhead(16, 64, 1, 16, seed=5)
    L_or, S_or, ld_or = O.selinv(M)
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=5.0).upload(M)
    try:
        assert S.stiles_workspace_bytes(st.h)[2] <= S.NOALLOC_SCRATCH_BYTES
        st.factor_selinv()
        torch.cuda.synchronize()
        assert st.status()[0] == S.STILES_OK
        L_ref, S_ref, ld_ref = st.L_tiles(), st.sigma_tiles(), st.logdet()
        for call in range(2):
            L2 = torch.full_like(st.L, float("nan"))
            S2 = torch.full_like(st.S, float("nan"))
            S.stiles_factor_selinv_noalloc(st.h, st.A.data_ptr(), L2.data_ptr(), S2.data_ptr(), st.stream_ptr())
            torch.cuda.synchronize()
            code, info, done = st.status()
            assert code == S.STILES_OK, (call, code, info)
            rc, ld = S.stiles_logdet(st.h)
            assert rc == S.STILES_OK
            Lg = st.layout.unpack(L2.cpu().numpy())
            Sg = st.layout.unpack(S2.cpu().numpy())
            assert rel_err(Lg, L_ref) < FP64_TOL, call
            assert rel_err(Sg, S_ref) < FP64_TOL, call
            assert abs(ld - ld_ref) < FP64_TOL * abs(ld_ref), call
            # and against the oracle directly (the same bar as every FP64 parity test)
            assert rel_err(Lg, L_or) < FP64_TOL, call
            assert rel_err(Sg, S_or) < FP64_TOL, call
            assert abs(ld - ld_or) < FP64_TOL * abs(ld_or), call
    finally:
        st.close()


@pytest.mark.gpu
def test_noalloc_rejects_shapes_beyond_the_array():
    S = need_gpu()
    import torch
    # scratch of this shape: about 2 x 8 x 64 x 1024^2 bytes of tiles, far above 64 MiB
    st = S.Stiles(64, 1024, 1, 8)
    try:
        assert S.stiles_workspace_bytes(st.h)[2] > S.NOALLOC_SCRATCH_BYTES
        A = torch.zeros(8, dtype=torch.float64, device="cuda")
        with pytest.raises(S.StilesError) as e:
            S.stiles_factor_selinv_noalloc(st.h, A.data_ptr(), st.L.data_ptr(), st.S.data_ptr(), 0)
        assert e.value.code == S.STILES_ERR_TOO_LARGE
    finally:
        st.close()
