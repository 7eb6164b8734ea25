"""Failure detection on the device, without a fault.

Every wait of the panel kernel's grid barrier is bounded: after the limit
(HPLGB_WAIT_TIMEOUT_MS, 2 s by default) the waiting CTA records DEV_TIMEOUT in
the library's device error word and returns, the other CTAs see the record and
return too, and hpl_sync_check() reports HPL_ERR_TIMEOUT (-103).  The test knob
HPLGB_TEST_EXTRA_ARRIVAL=1 makes every barrier wait for one arrival more than
the grid makes (an arrival nothing will make), so the first wait of each launch
runs out.  Nothing faults, traps or spins without a bound; the context stays
usable, which the test checks by factoring a system with the oracle's pivots
right afterwards on the same stream.
"""
from __future__ import annotations

import time

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def H():
    import __graft_entry__ as g
    g.build()
    import paper_2304_10397_gb300 as H
    assert torch.cuda.is_available()
    H.load_library()
    return H


def test_expired_barrier_wait_is_reported_and_the_context_recovers(H, monkeypatch):
    H.sync_check()  # nothing recorded before
    m, w = 4096, 48  # three base launches (widths 16, 8 ... as the recursion splits)
    A = H.colmajor(m, w)
    A.uniform_(-0.5, 0.5)
    ipiv = (torch.arange(w, dtype=torch.int32, device="cuda") + 1)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("HPLGB_WAIT_TIMEOUT_MS", "20")
    monkeypatch.setenv("HPLGB_TEST_EXTRA_ARRIVAL", "1")
    t0 = time.perf_counter()
    H.panel_getrf(A, ipiv=ipiv, info=info)  # the launches themselves succeed
    with pytest.raises(H.HplError) as exc:
        H.sync_check()
    elapsed = time.perf_counter() - t0
    assert exc.value.code == H.HPL_ERR_TIMEOUT
    # the first wait ran out after about 20 ms; later launches saw the record
    # and returned at once: well under the 2 s default limit per launch
    assert elapsed < 1.5, elapsed
    monkeypatch.delenv("HPLGB_TEST_EXTRA_ARRIVAL")
    monkeypatch.delenv("HPLGB_WAIT_TIMEOUT_MS")
    H.sync_check()  # the record was cleared by the check that reported it

    # the same stream and context factor a system correctly right afterwards
    n, nb, seed = 1024, 128, 42
    Ad, bd = H.generate(n, seed)
    piv, inf = H.getrf(Ad, nb)
    x = bd.clone()
    H.getrs("N", Ad, piv, x)
    H.sync_check()
    res = H.residual(n, seed, x)
    Ah, bh = O.generate(n, seed)
    gp = piv.cpu().numpy()[:n]
    _, oipiv, oinfo, st, _ = O.getrf(Ah, replay=gp, rtol=1e-13)
    assert st == 0 and np.array_equal(oipiv, gp)
    assert int(inf.item()) == 0 and res[0] < 16


def test_no_alloc_entry_reports_an_expired_wait_in_info(H, monkeypatch):
    m, w = 2048, 32
    A = H.colmajor(m, w)
    A.uniform_(-0.5, 0.5)
    ipiv = (torch.arange(w, dtype=torch.int32, device="cuda") + 1)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    monkeypatch.setenv("HPLGB_WAIT_TIMEOUT_MS", "20")
    monkeypatch.setenv("HPLGB_TEST_EXTRA_ARRIVAL", "1")
    H.panel_getrf_noalloc(A, ipiv, info)
    torch.cuda.synchronize()
    monkeypatch.delenv("HPLGB_TEST_EXTRA_ARRIVAL")
    monkeypatch.delenv("HPLGB_WAIT_TIMEOUT_MS")
    assert int(info.item()) == -1
    # the no-alloc path keeps its own error word, cleared at its next call
    H.sync_check()
    A.uniform_(-0.5, 0.5)
    H.panel_getrf_noalloc(A, ipiv, info)
    torch.cuda.synchronize()
    assert int(info.item()) == 0
