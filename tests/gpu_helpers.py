"""Shared helpers of the GPU tests: run the CUDA path through the C ABI and
compare with the oracle."""
import numpy as np
import pytest

FP64_TOL = 1e-10  # max |GPU - oracle| / max |oracle| over selected entries (FP64 target)


def need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2504_19171_gb300 import build
    build.build()
    from paper_2504_19171_gb300 import stiles
    return stiles


def rel_err(got: dict, ref: dict) -> float:
    num = max(np.abs(got[k] - ref[k]).max(initial=0.0) for k in ref)
    den = max(np.abs(ref[k]).max(initial=0.0) for k in ref)
    return num / den if den > 0 else num


def run_gpu(M, mode="fused", budget_s=5.0, precision=0):
    """Factor and invert M on the GPU. Returns (L tiles, Sigma tiles,
    logdet, (code, info, done))."""
    S = need_gpu()
    import torch
    st = S.Stiles(M.nt, M.b, M.w, M.a, wait_budget_s=budget_s, precision=precision).upload(M)
    try:
        if mode == "fused":
            st.factor_selinv()
        elif mode in ("split", "inplace"):
            st.factor(inplace=(mode == "inplace"))
            fstatus = st.status()
            st.selinv()
        else:
            raise ValueError(mode)
        torch.cuda.synchronize()
        status = st.status()
        if mode != "fused" and fstatus[0] != 0:
            status = fstatus
        ld = st.logdet() if status[0] == 0 else float("nan")
        return st.L_tiles(), st.sigma_tiles(), ld, status
    finally:
        st.close()
