"""Request server with continuous batching: requests of different shapes and
values admitted while others run; every result against the oracle, the same
request bit-identical alone and in the mix, per-request NOT_SPD, admission
by memory footprint (BUSY, then admitted after a release)."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from paper_2504_19171_gb300 import workloads as W
from tests.gpu_helpers import FP64_TOL, need_gpu, rel_err

POOL = [(6, 64, 1, 16), (5, 100, 2, 37), (9, 40, 3, 0)]


def _server(S, data_bytes=None, max_requests=16, precision=0, pool=POOL):
    import torch
    bases = [W.sweep_base(*sh, seed=20 + m) for m, sh in enumerate(pool)]
    need = max(3 * S.PackedLayout(*sh).doubles * 8 + 3 * 256 for sh in pool)
    srv = S.StilesServer(pool, data_bytes or 24 * need, max_requests=max_requests, precision=precision)
    for m, (M, rb, ra) in enumerate(bases):
        lay = srv.layouts[m]
        flat = torch.from_numpy(lay.pack(M.tiles, np.zeros(lay.doubles)))
        srv.set_base(m, flat, torch.from_numpy(rb), torch.from_numpy(ra))
    srv.start(60.0)
    return srv


def _wait(srv, want, timeout=30.0):
    done = {}
    t0 = time.time()
    while len(done) < want:
        for r, tag in srv.poll():
            done[tag] = r
        if time.time() - t0 > timeout:
            raise AssertionError(f"only {len(done)} of {want} requests completed")
        time.sleep(0.001)
    return done


def _sigma(srv, r, shape):
    import torch
    out = torch.empty(srv.layouts[shape].doubles, dtype=torch.float64)
    srv.sigma(r, out)
    return srv.layouts[shape].unpack(out.numpy())


@pytest.mark.gpu
def test_serve_alone_and_in_mix():
    S = need_gpu()
    srv = _server(S)
    try:
        # alone
        r = srv.submit(1, 0.8, 0.7, tag=0)
        assert r is not None
        done = _wait(srv, 1)
        alone = _sigma(srv, done[0], 1)
        assert srv.result(done[0])[0] == S.STILES_OK
        srv.release(done[0])
        # in a mix: arrivals while others run, the same request among them
        reqs = [(0, 1.5, 0.9), (2, 0.3, 0.5), (1, 0.8, 0.7), (0, 4.0, 0.95), (2, 9.0, 0.6), (1, 0.1, 0.99),
                (0, 0.6, 0.55), (2, 2.0, 0.8)]
        for tag, (shape, tau, rho) in enumerate(reqs, start=1):
            assert srv.submit(shape, tau, rho, tag=tag) is not None
        done = _wait(srv, len(reqs))
        for tag, (shape, tau, rho) in enumerate(reqs, start=1):
            r = done[tag]
            code, info, ld = srv.result(r)
            assert code == S.STILES_OK
            sig = _sigma(srv, r, shape)
            A = W.sweep_arrowhead(*POOL[shape], tau, rho, seed=20 + shape)
            _, Sr, ldr = O.selinv(A)
            assert rel_err(sig, Sr) < FP64_TOL, tag
            assert abs(ld - ldr) < FP64_TOL * max(1.0, abs(ldr))
            if (shape, tau, rho) == (1, 0.8, 0.7):
                assert all(np.array_equal(sig[k], alone[k]) for k in alone)
            srv.release(r)
        assert srv.stop() == S.STILES_OK
    finally:
        srv.close()


@pytest.mark.gpu
def test_serve_not_spd_request_is_isolated():
    S = need_gpu()
    srv = _server(S)
    try:
        assert srv.submit(0, -30.0, 0.9, tag=1) is not None  # tau far below zero: indefinite
        assert srv.submit(2, 1.0, 0.9, tag=2) is not None
        done = _wait(srv, 2)
        code, info, ld = srv.result(done[1])
        assert code == S.STILES_ERR_NOT_SPD and info >= 1 and np.isnan(ld)
        assert srv.result(done[2])[0] == S.STILES_OK
        for r in done.values():
            srv.release(r)
        assert srv.stop() == S.STILES_OK
    finally:
        srv.close()


@pytest.mark.gpu
def test_serve_admission_by_memory():
    S = need_gpu()
    pool = [(6, 64, 1, 16)]
    probe = S.StilesServer(pool, 1 << 20, max_requests=4)
    per = probe.request_bytes(0)
    probe.close()
    srv = _server(S, data_bytes=2 * per + 1024, pool=pool)
    try:
        a = srv.submit(0, 1.0, 0.5, tag=1)
        b = srv.submit(0, 2.0, 0.5, tag=2)
        assert a is not None and b is not None
        assert srv.submit(0, 3.0, 0.5, tag=3) is None  # no memory now
        done = _wait(srv, 2)
        srv.release(done[1])
        assert srv.submit(0, 3.0, 0.5, tag=3) is not None  # admitted after the release
        done.update(_wait(srv, 1))
        for tag in (2, 3):
            srv.release(done[tag])
        assert srv.stop() == S.STILES_OK
    finally:
        srv.close()


@pytest.mark.gpu
def test_serve_emulated_fp64():
    """Served requests in the emulated-FP64 mode against the oracle (the
    emulated mode's 1e-12 target)."""
    S = need_gpu()
    srv = _server(S, precision=S.STILES_EMU64)
    try:
        reqs = [(0, 0.9, 0.8), (1, 2.0, 0.6), (2, 0.5, 0.95)]
        for tag, (shape, tau, rho) in enumerate(reqs):
            assert srv.submit(shape, tau, rho, tag=tag) is not None
        done = _wait(srv, len(reqs))
        for tag, (shape, tau, rho) in enumerate(reqs):
            r = done[tag]
            assert srv.result(r)[0] == S.STILES_OK
            A = W.sweep_arrowhead(*POOL[shape], tau, rho, seed=20 + shape)
            _, Sr, _ = O.selinv(A)
            assert rel_err(_sigma(srv, r, shape), Sr) < 1e-12
            srv.release(r)
        assert srv.stop() == S.STILES_OK
    finally:
        srv.close()


@pytest.mark.gpu
def test_serve_explicit_values():
    """A request carrying its own A (copied in before it joins the kernel)
    against the oracle, mixed with sweep requests."""
    S = need_gpu()
    srv = _server(S)
    try:
        A1 = W.random_arrowhead(*POOL[1], seed=77)
        flat = srv.layouts[1].pack(A1.tiles, np.zeros(srv.layouts[1].doubles))
        assert srv.submit(0, 1.2, 0.8, tag=0) is not None
        assert srv.submit_values(1, flat, tag=1) is not None
        assert srv.submit(2, 0.7, 0.9, tag=2) is not None
        done = _wait(srv, 3)
        r = done[1]
        code, _, ld = srv.result(r)
        assert code == S.STILES_OK
        _, Sr, ldr = O.selinv(A1)
        assert rel_err(_sigma(srv, r, 1), Sr) < FP64_TOL
        assert abs(ld - ldr) < FP64_TOL * max(1.0, abs(ldr))
        for q in done.values():
            srv.release(q)
        assert srv.stop() == S.STILES_OK
    finally:
        srv.close()
