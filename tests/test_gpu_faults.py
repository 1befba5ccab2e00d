"""Failure detection without a GPU fault: every device-side wait is bounded,
so a wait limit of one poll makes the sweep give up.  The status word
reports ILU_ETIMEOUT, the handle refuses further work, and the CUDA context
stays usable (a fresh handle sweeps correctly afterwards)."""
import numpy as np
import pytest

import seeded_inputs as si

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2210_15280_gb300 as g
    g.build()
    return g


@pytest.mark.parametrize("kernel", ["SLAB", "BAND"])
def test_bounded_wait_reports_timeout(g, kernel):
    level = 6
    P = si.macro_tet(7)
    k = getattr(g, "KERNEL_" + kernel)
    b = torch.tensor(si.rhs(level, 8), dtype=torch.float64, device="cuda")
    timed_out = False
    for attempt in range(5):  # a wait that never has to wait cannot run out
        t = g.Tet(P, level, poly_degree=4, precision=g.MIXED, kernel=k, max_wait_spins=1)
        x = torch.zeros_like(b)
        try:
            t.smooth(x, b, 2, norms=True)  # norms: the call reads the status word
        except g.IluError as e:
            assert e.status == g.ILU_ETIMEOUT, str(e)
            timed_out = True
            with pytest.raises(g.IluError) as e2:
                t.smooth(x, b, 1)
            assert e2.value.status == g.ILU_ECUDA  # failed handle: destroy it
            t.close()
            break
        t.close()
    assert timed_out
    # the context is intact: a normal handle gives the normal result
    ref = g.Tet(P, level, poly_degree=4, precision=g.MIXED, kernel=k)
    x1 = torch.zeros_like(b)
    n1 = ref.smooth(x1, b, 2, norms=True)
    ref2 = g.Tet(P, level, poly_degree=4, precision=g.MIXED, kernel=k)
    x2 = torch.zeros_like(b)
    n2 = ref2.smooth(x2, b, 2, norms=True)
    assert np.array_equal(n1, n2) and torch.equal(x1, x2)
    assert np.isfinite(x1.cpu().numpy()).all()


def test_batch_timeout_is_reported(g):
    """Slab-kernel tets (the packed kernels never wait on another CTA, so a
    batch of packed tets has no wait to run out)."""
    level = 6
    tets = [g.Tet(si.macro_tet(20 + i), level, poly_degree=4, precision=g.MIXED, kernel=g.KERNEL_SLAB)
            for i in range(3)]
    b = [torch.tensor(si.rhs(level, 30 + i), dtype=torch.float64, device="cuda") for i in range(3)]
    hit = False
    for attempt in range(5):
        B = g.Batch(tets, max_wait_spins=1)
        x = [torch.zeros_like(v) for v in b]
        try:
            B.smooth(x, b, 1)
        except g.IluError as e:
            assert e.status == g.ILU_ETIMEOUT
            hit = True
            with pytest.raises(g.IluError):
                B.smooth(x, b, 1)  # a failed batch refuses work
            B.close()
            break
        B.close()
    assert hit
    # the tets themselves are unaffected
    x = torch.zeros_like(b[0])
    tets[0].smooth(x, b[0], 1)
    assert np.isfinite(x.cpu().numpy()).all()
