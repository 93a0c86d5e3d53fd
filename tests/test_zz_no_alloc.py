"""The allocation-free batched distance map (td_edm_batched_noalloc), called through the C ABI.

Some callers cannot allocate device memory -- a serving process whose memory pool already holds
all the memory it may use, a plugin inside a framework that owns every device allocation, or a
latency-bound loop where an allocation and the synchronisation it brings are not acceptable --
so this entry point keeps its launch plan in a fixed device array inside the library instead of
a caller workspace.  Its output must equal the workspace-based td_edm_batched bit for bit, call
after call (the second call below plans a different batch into the same array), and the CPU
oracle within the FP32 distance tolerance.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import oracle
from paper_1308_1419_gb300 import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_1308_1419_gb300 import td  # noqa: E402

RTOL = 2e-6  # the FP32 distance-map tolerance used throughout the tests
MAX_PROBLEMS = 1024  # the fixed array's capacity, as td.h states it


def _call_c_abi(ns, ds, x, out, rho):
    nh = np.ascontiguousarray(ns, dtype=np.uint32)
    dh = np.ascontiguousarray(ds, dtype=np.uint32)
    cfg = td.td_batched_config(rho, 0)
    st = td.td_launch_stats()
    f = td.lib.td_edm_batched_noalloc
    f.restype = C.c_int
    f.argtypes = [C.c_uint32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                  C.POINTER(td.td_batched_config), C.POINTER(td.td_launch_stats), C.c_void_p]
    rc = f(len(nh), nh.ctypes.data_as(C.c_void_p), dh.ctypes.data_as(C.c_void_p), x.data_ptr(), out.data_ptr(),
           C.byref(cfg), C.byref(st), torch.cuda.current_stream().cuda_stream)
    return rc, st


def _check_batch(ns, ds, xh, rho):
    x = torch.from_numpy(xh).cuda()
    ref, _, _ = td.td_edm_batched(ns, ds, x, config=(rho, 0))
    _, os_ = td.batched_sizes(ns, ds)
    out = torch.full((os_,), float("nan"), dtype=torch.float32, device="cuda")
    rc, st = _call_c_abi(ns, ds, x, out, rho)
    assert rc == 0, td.lib.td_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    assert np.array_equal(got.view(np.uint32), ref[:os_].cpu().numpy().view(np.uint32))  # bit for bit
    want = oracle.edm_batched(xh, ns, ds)
    assert np.all(np.abs(got.astype(np.float64) - want) <= RTOL * want + 1e-30)
    assert st.launches == 1


def test_noalloc_matches_workspace_form_two_calls_in_a_row():
    batches = [synth.batched_problems(nprob=48, nmin=1, ratio=300.0, dims=(1, 3, 16, 64), seed=21),
               synth.batched_problems(nprob=300, nmin=8, ratio=64.0, dims=(3, 16, 64), seed=22)]
    for (ns, ds, xh), rho in zip(batches, (64, 128)):
        _check_batch(ns, ds, xh, rho)


def test_noalloc_at_its_maximum_problem_count():
    """Exactly the array's capacity: every plan entry in use, and the whole prefix array still
    staged in the kernel's shared memory."""
    ns, ds, xh = synth.batched_problems(nprob=MAX_PROBLEMS, nmin=1, ratio=40.0, dims=(1, 3, 8), seed=23)
    _check_batch(ns, ds, xh, 64)


def test_noalloc_rejects_more_than_its_maximum():
    ns = np.full(MAX_PROBLEMS + 1, 4, dtype=np.uint32)
    ds = np.full(MAX_PROBLEMS + 1, 3, dtype=np.uint32)
    x = torch.zeros(int(ns.sum()) * 3, device="cuda")
    out = torch.zeros(int((ns * (ns + 1) // 2).sum()), device="cuda")
    rc, _ = _call_c_abi(ns, ds, x, out, 64)
    assert rc == 1
