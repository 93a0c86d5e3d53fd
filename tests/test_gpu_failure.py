"""Failure detection on the device without a fault: the bounded mbarrier wait the Gram pipeline
uses is made to run out (a barrier nothing arrives on); the kernel records the timeout and
returns, the host reads TD_ERR_TIMEOUT, and the context stays usable for the next launch."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402


def test_wait_completes_when_the_phase_completes():
    ns = td.td_wait_selftest(True, 10**8)
    assert ns < 10**8


@pytest.mark.parametrize("limit_ns", [10**5, 10**7])
def test_wait_runs_out_and_reports_timeout(limit_ns):
    with pytest.raises(td.TDError) as e:
        td.td_wait_selftest(False, limit_ns)
    assert e.value.status == 4 and "ran out" in str(e.value)
    # The wait gave up after its limit, not much later (the time check runs every 64 polls).
    ws = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(td.TDError):
        td.td_wait_selftest(False, limit_ns, ws)
    rec = ws.cpu().numpy()
    assert rec[0] == 1 and limit_ns <= rec[1] < limit_ns + 5 * 10**8


def test_context_usable_after_timeout():
    with pytest.raises(td.TDError):
        td.td_wait_selftest(False, 10**6)
    N, rho = 3000, 16
    out, _ = td.td_map_probe("LTM", "persistent", N, rho)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32)[:td.td_tri_size(N)], oracle.probe(N))
    assert td.td_wait_selftest(True, 10**6) < 10**6 + 5 * 10**8


def test_completed_phase_passes_at_the_shortest_limit():
    # The phase completes before the wait starts, so even a 1 us limit sees it.
    for _ in range(3):
        assert td.td_wait_selftest(True, 1000) < 10**9
